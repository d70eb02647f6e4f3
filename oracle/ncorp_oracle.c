/*
 * ncorp_oracle.c -- plain, slow, FP64 CPU oracle for the falcON step of
 * Couturier, Quillen & Nakajima, "NcorpiON: a O(N) software for N-body
 * integration in collisional and fragmenting systems" (arXiv 2310.20374).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file: only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code with the CUDA library.
 *
 * Compiled with -O2 -ffp-contract=off (no fused multiply-add, no fast-math),
 * so every floating-point expression below is evaluated exactly in the
 * order written.
 *
 * What it computes (each function cites the passage it follows):
 *   - direct O(N^2) mutual gravity (Sect. 3.2)                   pinned
 *   - central-body and distant-star accelerations (App. B.1, B.3) pinned
 *   - root cube, quantisation and 3-D Hilbert keys (Sect. 3.4.6)  pinned
 *   - opening angle theta(M) (Dehnen 2002, Eq. 13; cited, not printed,
 *     in Sect. 3.4.3)                                              pinned
 *   - octree (Sect. 3.4.1), tree climbing for gravity and for collisions
 *     (Sect. 3.4.2, Eqs. center/rmax/rcrit and expansion_center/rmax_2/
 *     rcrit_2, corner cap)                                          pinned
 *   - Green-function derivative tensors (Eq. gradient), P2M
 *     (Eq. multipole_moment), M2M (App. C), symmetric M2L
 *     (Eq. phi_expanded and the A<->B relation of Sect. 3.4.3), L2L/L2P
 *     (Eq. shifting) with full 3^n tensors (no symmetric compression)  pinned
 *   - the dual tree walk (Algorithm TreeWalk, Sect. 3.4.5)           pinned
 *   - the standard tree code (Algorithm StandardTree, Sect. 3.4.4)
 *     with M2P (the m = 1 term of Eq. phi_expanded at a point), and
 *     its collision search                                            pinned
 *   - the collision predicate (Sect. 3.1), brute force and tree-based  pinned
 *   - the SBAB1 kick-drift-kick step with merged kicks (Sect. 4.1)    pinned
 *   - elastic and inelastic collision resolution (Sect. 5.1, 5.2)     pinned
 *
 * Readings of points the paper leaves open (numbered as in the design
 * notes): root cube and quantisation; Skilling's Hilbert curve; ties in the
 * sort by (key, index); never split a leaf in TreeWalk; 36 self pairs
 * including (a,a); "well separated" as (rcA+rcB)^2 <= |sA-sB|^2; no
 * softening; collision pruning with a 2^-40 relative margin; the corner
 * cap computed on the cell cube widened by L*2^-48; the moonlet mean of
 * Eq. center weighted by child counts; theta(M) solved by 12 bisection
 * steps and 4 Newton steps without libm; one impact per moonlet per step,
 * pairs resolved in increasing (dt_c, i, j), the rest of the step travelled
 * at the new velocity.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXP 6
#define OR_BITS 21

typedef struct {
    double G, central_mass;
    int p;                  /* expansion order, 1..6 */
    double theta_min;       /* theta at the root */
    int leaf_size;          /* s: a cell with more than s moonlets is split */
    int64_t n_cs, n_cc_pre, n_cc_post;   /* gravity TreeWalk thresholds */
    int64_t c_cs, c_cc_pre, c_cc_post;   /* collision TreeWalk thresholds */
    double star_mass, star_a, star_obliquity, time; /* App. B.3; star_mass = 0 disables */
    int m2m_direct;         /* 1: parent multipoles by direct P2M over all members */
    int brute_collisions;   /* KDK: 1 = brute force pairs, 0 = tree */
    double central_radius, central_J2;   /* App. B.2 equatorial bulge; J2 = 0 disables */
    double resolve_f;       /* KDK: 0 = pairs reported only; 1..2 = resolved with this f (Sect. 5) */
    int64_t n_cb_pre, n_cb_post;         /* StandardTree thresholds (Sect. 3.4.4), gravity */
    int64_t c_cb_pre, c_cb_post;         /* StandardTree thresholds, collision search */
} or_params;

/* statistics, int64 slots */
enum { ST_CELLS, ST_LEAVES, ST_DEPTH, ST_M2L, ST_P2P_PAIRS, ST_P2P_SELF, ST_P2P_INTER,
       ST_COL_PAIRS, ST_COL_SELF, ST_COL_TESTS, ST_COL_FOUND, ST_NSTAT = 16 };

/* ------------------------------------------------------------------------ */
/* Small vector helpers (fixed evaluation order).                           */
/* ------------------------------------------------------------------------ */
static double norm3(const double d[3]) { return sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]); }
static double dot3(const double a[3], const double b[3]) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }

/* ------------------------------------------------------------------------ */
/* Root cube, quantisation, Hilbert keys (Sect. 3.4.6).                     */
/* Root: centre = midpoint of the bounding box, side L = the smallest power */
/* of two >= (max extent)(1 + 2^-20).  q = floor((x - x_lo) 2^21 / L).     */
/* ------------------------------------------------------------------------ */
void or_root(int64_t n, const double *pos, double root[4])
{
    double lo[3], hi[3];
    for (int k = 0; k < 3; k++) { lo[k] = n > 0 ? pos[k] : 0.0; hi[k] = lo[k]; }
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < 3; k++) {
            double v = pos[3 * i + k];
            if (v < lo[k]) lo[k] = v;
            if (v > hi[k]) hi[k] = v;
        }
    double ext = 0.0;
    for (int k = 0; k < 3; k++) { double e = hi[k] - lo[k]; if (e > ext) ext = e; }
    double t = ext * (1.0 + 0x1p-20);
    double L = 1.0;
    if (t > 0.0) {
        while (L < t) L *= 2.0;
        while (L * 0.5 >= t) L *= 0.5;
    }
    for (int k = 0; k < 3; k++) root[k] = (lo[k] + hi[k]) * 0.5 - L * 0.5;
    root[3] = L;
}

static uint32_t quantise(double x, double xlo, double scale)
{
    double f = floor((x - xlo) * scale);
    if (f < 0.0) f = 0.0;
    if (f > (double)((1u << OR_BITS) - 1)) f = (double)((1u << OR_BITS) - 1);
    return (uint32_t)f;
}

/* Skilling's transpose-form Hilbert index (J. Skilling, "Programming the
 * Hilbert curve", AIP Conf. Proc. 707, 381 (2004)), restated for 3 axes:
 * undo the excess work of the Gray-code reflection/exchange per bit plane,
 * then Gray-encode; the key interleaves the transposed bits, MSB first,
 * axis 0 first. */
uint64_t or_hilbert_key(uint32_t x, uint32_t y, uint32_t z, int bits)
{
    uint32_t X[3] = {x, y, z};
    uint32_t top = 1u << (bits - 1);
    for (uint32_t Q = top; Q > 1; Q >>= 1) {
        uint32_t P = Q - 1;
        for (int i = 0; i < 3; i++) {
            if (X[i] & Q) {
                X[0] ^= P;                       /* reflect */
            } else {
                uint32_t t = (X[0] ^ X[i]) & P;  /* exchange low bits of axis 0 and i */
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    uint32_t t = 0;
    for (uint32_t Q = top; Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    for (int i = 0; i < 3; i++) X[i] ^= t;
    uint64_t key = 0;
    for (int b = bits - 1; b >= 0; b--)
        for (int i = 0; i < 3; i++) key = (key << 1) | ((X[i] >> b) & 1u);
    return key;
}

/* keys and quantised coordinates of every moonlet */
void or_keys(int64_t n, const double *pos, double root[4], uint32_t *q, uint64_t *keys)
{
    or_root(n, pos, root);
    double scale = (double)(1u << OR_BITS) / root[3];
    for (int64_t i = 0; i < n; i++) {
        for (int k = 0; k < 3; k++) q[3 * i + k] = quantise(pos[3 * i + k], root[k], scale);
        keys[i] = or_hilbert_key(q[3 * i], q[3 * i + 1], q[3 * i + 2], OR_BITS);
    }
}

/* ------------------------------------------------------------------------ */
/* Opening angle theta(M) (Dehnen 2002, Eq. 13):                            */
/*   theta^5/(1-theta)^2 = [theta_min^5/(1-theta_min)^2] (M/M_tot)^(-1/3),  */
/* i.e. the root in [theta_min, 1) of the increasing                         */
/*   f(theta) = theta^15 M - K^3 M_tot (1-theta)^6:                          */
/* 12 bisection steps, then 4 Newton steps kept inside the final bracket,    */
/* with + - x / only (no libm), so that any IEEE implementation evaluating   */
/* the same expressions in the same order gets the same bits.                */
/* ------------------------------------------------------------------------ */
double or_theta(double M, double Mtot, double theta_min)
{
    double t2 = theta_min * theta_min, t4 = t2 * t2, t5 = t4 * theta_min;
    double u = 1.0 - theta_min, u2 = u * u;
    double K = t5 / u2;
    double K3 = (K * K) * K;
    double rhs = K3 * Mtot;
    double lo = theta_min, hi = 1.0;
    for (int it = 0; it < 12; it++) {
        double mid = (lo + hi) * 0.5;
        double m2 = mid * mid, m3 = m2 * mid, m6 = m3 * m3, m12 = m6 * m6, m15 = m12 * m3;
        double w = 1.0 - mid, w2 = w * w, w3 = w2 * w, w6 = w3 * w3;
        double f = m15 * M - rhs * w6;
        if (f > 0.0) hi = mid; else lo = mid;
    }
    double th = (lo + hi) * 0.5;
    for (int it = 0; it < 4; it++) {
        double w = 1.0 - th;
        double q2 = th * th, q3 = q2 * th, q6 = q3 * q3, q12 = q6 * q6, q14 = q12 * q2, q15 = q14 * th;
        double w2 = w * w, w3 = w2 * w, w5 = w3 * w2, w6 = w3 * w3;
        double f = q15 * M - rhs * w6;
        double fp = (15.0 * q14) * M + (6.0 * rhs) * w5;
        double nt = th - f / fp;
        if (nt < lo) nt = lo;
        if (nt > hi) nt = hi;
        th = nt;
    }
    return th;
}

/* ------------------------------------------------------------------------ */
/* Full Cartesian tensors: order n stored as 3^n doubles, flat index        */
/* t = i1 3^(n-1) + ... + in (first index most significant).  Packed sets   */
/* of orders 0..P keep order n at offset (3^n - 1)/2.                       */
/* ------------------------------------------------------------------------ */
static const int POW3[9] = {1, 3, 9, 27, 81, 243, 729, 2187, 6561};
static int OFF(int n) { return (POW3[n] - 1) / 2; }
static const double INV_FACT[8] = {1.0, 1.0, 0.5, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0, 1.0 / 720.0, 1.0 / 5040.0};
static int digit(int t, int n, int k) { return (t / POW3[n - 1 - k]) % 3; } /* k-th index of tuple t */

/* d^(n) = n-fold outer product of d with itself */
static void outer_power(const double d[3], int n, double *out)
{
    for (int t = 0; t < POW3[n]; t++) {
        double v = 1.0;
        for (int k = 0; k < n; k++) v *= d[digit(t, n, k)];
        out[t] = v;
    }
}

/* ---- Green-function derivatives (Eq. gradient) ------------------------
 * (nabla^(n) g)_{i1..in} = d/dR_in (nabla^(n-1) g)_{i1..i(n-1)}, g = 1/R.
 * Every component has the form P(R)/|R|^(2n+1) with P homogeneous of degree
 * n; differentiating gives P' = |R|^2 dP/dR_j - (2n+1) R_j P.  The integer
 * polynomials are generated once by applying that rule literally. */
#define OR_DMAX 6
static int mono_count(int n) { return (n + 1) * (n + 2) / 2; }
static int mono_idx(int n, int a, int b) { int k = n - a; int c = k - b; return k * (k + 1) / 2 + c; }
static double *g_poly[OR_DMAX + 1];   /* g_poly[n][t * mono_count(n) + mono] */
static int g_poly_ready = 0;

static void build_polys(void)
{
    if (g_poly_ready) return;
    g_poly[0] = (double *)calloc(1, sizeof(double));
    g_poly[0][0] = 1.0;
    for (int n = 0; n < OR_DMAX; n++) {
        int mc = mono_count(n), mc1 = mono_count(n + 1);
        g_poly[n + 1] = (double *)calloc((size_t)POW3[n + 1] * mc1, sizeof(double));
        for (int t = 0; t < POW3[n]; t++) {
            const double *P = g_poly[n] + (size_t)t * mc;
            for (int j = 0; j < 3; j++) {
                double *Q = g_poly[n + 1] + (size_t)(t * 3 + j) * mc1;
                for (int a = n; a >= 0; a--)
                    for (int b = n - a; b >= 0; b--) {
                        int c = n - a - b;
                        double k = P[mono_idx(n, a, b)];
                        if (k == 0.0) continue;
                        int e[3] = {a, b, c};
                        /* |R|^2 * dP/dR_j */
                        if (e[j] > 0) {
                            double kd = k * e[j];
                            int f[3] = {a, b, c};
                            f[j] -= 1;
                            for (int s = 0; s < 3; s++) {
                                int g2[3] = {f[0], f[1], f[2]};
                                g2[s] += 2;
                                Q[mono_idx(n + 1, g2[0], g2[1])] += kd;
                            }
                        }
                        /* -(2n+1) R_j P */
                        int h[3] = {a, b, c};
                        h[j] += 1;
                        Q[mono_idx(n + 1, h[0], h[1])] -= (double)(2 * n + 1) * k;
                    }
            }
        }
    }
    g_poly_ready = 1;
}

/* D^(n)(R) as a full 3^n tensor */
void or_dtensor(int n, const double R[3], double *out)
{
    build_polys();
    double r2 = (R[0] * R[0] + R[1] * R[1]) + R[2] * R[2];
    double r = sqrt(r2);
    double inv = 1.0 / r, scale = inv;
    for (int k = 0; k < n; k++) scale = scale * (inv * inv);
    double px[OR_DMAX + 1], py[OR_DMAX + 1], pz[OR_DMAX + 1];
    px[0] = py[0] = pz[0] = 1.0;
    for (int k = 1; k <= n; k++) { px[k] = px[k - 1] * R[0]; py[k] = py[k - 1] * R[1]; pz[k] = pz[k - 1] * R[2]; }
    double mono[64];
    for (int a = n; a >= 0; a--)
        for (int b = n - a; b >= 0; b--) mono[mono_idx(n, a, b)] = (px[a] * py[b]) * pz[n - a - b];
    int mc = mono_count(n);
    for (int t = 0; t < POW3[n]; t++) {
        const double *P = g_poly[n] + (size_t)t * mc;
        double v = 0.0;
        for (int m = 0; m < mc; m++) v += P[m] * mono[m];
        out[t] = v * scale;
    }
}

/* ---- P2M (Eq. multipole_moment): M^(n)(s) = sum_i mu_i (x_i - s)^(n),
 * packed orders 0..p-1 (order 1 is kept and is ~0 about the barycentre). */
void or_p2m(int p, int64_t k, const double *pos, const double *mu, const double s[3], double *out)
{
    int tot = OFF(p);
    memset(out, 0, sizeof(double) * tot);
    double tmp[729];
    for (int64_t i = 0; i < k; i++) {
        double d[3] = {pos[3 * i] - s[0], pos[3 * i + 1] - s[1], pos[3 * i + 2] - s[2]};
        for (int n = 0; n < p; n++) {
            outer_power(d, n, tmp);
            for (int t = 0; t < POW3[n]; t++) out[OFF(n) + t] += mu[i] * tmp[t];
        }
    }
}

/* ---- M2M (App. C): contribution of child b (moments m about s_b) to the
 * moments of its parent about s_B, Lambda = s_B - s_b, with m^(1) = 0:
 * every index position is taken either from m or from -Lambda; the sum
 * over all such subsets reproduces the closed forms listed for n <= 5. */
void or_m2m(int p, const double *m, const double sb[3], const double sB[3], double *out)
{
    double Lam[3] = {sB[0] - sb[0], sB[1] - sb[1], sB[2] - sb[2]};
    for (int n = 0; n < p; n++) {
        for (int t = 0; t < POW3[n]; t++) {
            int idx[8];
            for (int k = 0; k < n; k++) idx[k] = digit(t, n, k);
            double acc = 0.0;
            for (int S = 0; S < (1 << n); S++) {
                int ns = __builtin_popcount((unsigned)S);
                int rest = n - ns;
                if (rest == 1) continue;            /* dipole about the barycentre vanishes */
                double lam = 1.0;
                int rt = 0;
                for (int k = 0; k < n; k++) {
                    if (S & (1 << k)) lam *= Lam[idx[k]];
                    else rt = rt * 3 + idx[k];
                }
                double term = lam * m[OFF(rest) + rt];
                acc += (ns & 1) ? -term : term;
            }
            out[OFF(n) + t] += acc;
        }
    }
}

/* T^(m+n) contracted on its last n indices with V^(n): result of order m */
static void contract(const double *T, int m, int n, const double *V, double *out, double factor)
{
    for (int o = 0; o < POW3[m]; o++) {
        double acc = 0.0;
        const double *row = T + (size_t)o * POW3[n];
        for (int t = 0; t < POW3[n]; t++) acc += row[t] * V[t];
        out[o] += factor * acc;
    }
}

/* ---- symmetric M2L (Eq. phi_expanded; A<->B relation of Sect. 3.4.3):
 * R = s_A - s_B,
 *   C_A^(m) += sum_{n=0}^{p-m} (-1)^n/n! D^(n+m)(R) . M_B^(n)
 *   C_B^(m) += (-1)^m sum_{n=0}^{p-m} 1/n! D^(n+m)(R) . M_A^(n)
 * one D evaluation per pair; C packed by order (order 0 unused). */
void or_m2l(int p, const double sA[3], const double *MA, const double sB[3], const double *MB,
            double *CA, double *CB)
{
    double R[3] = {sA[0] - sB[0], sA[1] - sB[1], sA[2] - sB[2]};
    static double D[OR_DMAX + 1][729];
    for (int k = 1; k <= p; k++) or_dtensor(k, R, D[k]);
    for (int m = 1; m <= p; m++)
        for (int n = 0; n <= p - m; n++) {
            if (n == 1) continue;
            double sgnA = (n & 1) ? -INV_FACT[n] : INV_FACT[n];
            double sgnB = (m & 1) ? -INV_FACT[n] : INV_FACT[n];
            contract(D[n + m], m, n, MB + OFF(n), CA + OFF(m), sgnA);
            contract(D[n + m], m, n, MA + OFF(n), CB + OFF(m), sgnB);
        }
}

/* ---- L2L (Eq. shifting): C^(m)(s1) = sum_{n=0}^{p-m} 1/n! C^(m+n)(s0) . (s1-s0)^(n),
 * added into Cout. */
void or_l2l(int p, const double *Cin, const double s0[3], const double s1[3], double *Cout)
{
    double d[3] = {s1[0] - s0[0], s1[1] - s0[1], s1[2] - s0[2]};
    double pw[729];
    for (int m = 1; m <= p; m++)
        for (int n = 0; n <= p - m; n++) {
            outer_power(d, n, pw);
            contract(Cin + OFF(m + n), m, n, pw, Cout + OFF(m), INV_FACT[n]);
        }
}

/* ---- L2P: acceleration C^(1)(x) from C^(m)(s) (Eq. shifting with s1 = x) */
void or_l2p(int p, const double *C, const double s[3], const double x[3], double acc[3])
{
    double d[3] = {x[0] - s[0], x[1] - s[1], x[2] - s[2]};
    double pw[729];
    double out[3] = {0, 0, 0};
    for (int n = 0; n <= p - 1; n++) {
        outer_power(d, n, pw);
        contract(C + OFF(1 + n), 1, n, pw, out, INV_FACT[n]);
    }
    acc[0] += out[0];
    acc[1] += out[1];
    acc[2] += out[2];
}

/* ---- M2P: the field C^(1) of cell B's expansion at the point x, i.e. the
 * m = 1 term of Eq. phi_expanded for a target reduced to the point x:
 *   C^(1)(x) += sum_{n=0}^{p-1} (-1)^n/n! D^(n+1)(x - s_B) . M_B^(n). */
void or_m2p(int p, const double x[3], const double sB[3], const double *MB, double acc[3])
{
    double R[3] = {x[0] - sB[0], x[1] - sB[1], x[2] - sB[2]};
    static double D[729];
    for (int n = 0; n <= p - 1; n++) {
        if (n == 1) continue;
        or_dtensor(n + 1, R, D);
        contract(D, 1, n, MB + OFF(n), acc, (n & 1) ? -INV_FACT[n] : INV_FACT[n]);
    }
}

/* ------------------------------------------------------------------------ */
/* Direct gravity (Sect. 3.2) and external forces (App. B.1, B.3).          */
/* ------------------------------------------------------------------------ */
void or_direct_accel(int64_t n, const double *pos, const double *mass, double G,
                     int64_t nt, const int64_t *targets, double *acc)
{
    for (int64_t a = 0; a < nt; a++) {
        int64_t i = targets ? targets[a] : a;
        double s[3] = {0, 0, 0};
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double d[3] = {pos[3 * i] - pos[3 * j], pos[3 * i + 1] - pos[3 * j + 1], pos[3 * i + 2] - pos[3 * j + 2]};
            double r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
            if (r2 == 0.0) continue;                /* no softening; coincident pair skipped */
            double r = sqrt(r2);
            double f = (G * mass[j]) / (r2 * r);
            for (int k = 0; k < 3; k++) s[k] -= f * d[k];
        }
        for (int k = 0; k < 3; k++) acc[3 * a + k] = s[k];
    }
}

/* star position on its circular, inclined orbit (App. B.3) */
static void star_position(const or_params *P, double t, double rs[3])
{
    double nsun = sqrt(P->G * P->star_mass / (P->star_a * P->star_a * P->star_a));
    double lam = nsun * t;
    rs[0] = P->star_a * cos(lam);
    rs[1] = P->star_a * sin(lam) * cos(P->star_obliquity);
    rs[2] = P->star_a * sin(lam) * sin(P->star_obliquity);
}

/* central mass (App. B.1) + optional equatorial bulge of the central body
 * (App. B.2: a = G M_c R_c^2 J2 / r^5 [ (15 z^2 - 3 r^2) / (2 r^2) r - 3 z k ],
 * k the body's rotation axis = the frame's z axis) + optional quadrupole star
 * tide (App. B.3), added into acc */
void or_external_accel(const or_params *P, int64_t n, const double *pos, double t, double *acc)
{
    double rs[3] = {0, 0, 0}, rs2 = 0.0, ks = 0.0;
    int star = P->star_mass != 0.0;
    if (star) {
        star_position(P, t, rs);
        rs2 = dot3(rs, rs);
        ks = (P->G * P->star_mass) / (rs2 * sqrt(rs2));
    }
    for (int64_t i = 0; i < n; i++) {
        const double *x = pos + 3 * i;
        double r2 = (x[0] * x[0] + x[1] * x[1]) + x[2] * x[2];
        double r = sqrt(r2);
        double f = -(P->G * P->central_mass) / (r2 * r);
        for (int k = 0; k < 3; k++) acc[3 * i + k] += f * x[k];
        if (P->central_J2 != 0.0) {
            double q = P->G * P->central_mass * P->central_radius * P->central_radius * P->central_J2 / (r2 * r2 * r);
            double z2 = x[2] * x[2];
            double radial = q * (15.0 * z2 - 3.0 * r2) / (2.0 * r2);
            for (int k = 0; k < 3; k++) acc[3 * i + k] += radial * x[k];
            acc[3 * i + 2] -= 3.0 * q * x[2];
        }
        if (star) {
            double c = 3.0 * dot3(x, rs) / rs2;
            for (int k = 0; k < 3; k++) acc[3 * i + k] -= ks * (x[k] - c * rs[k]);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Collision predicate (Sect. 3.1).  dr = r1 - r2, dv = v1 - v2,            */
/* Delta = (dr.dv)^2 + dv^2 ((R1+R2)^2 - dr^2), dt_c = -(dr.dv + sqrt(Delta))/dv^2, */
/* collision iff Delta >= 0 and 0 <= dt_c <= dt.                            */
/* ------------------------------------------------------------------------ */
/* Time of impact: returns 1 and *tc when Delta >= 0 and dv^2 != 0. */
static int impact_time(const double x1[3], const double v1[3], double R1,
                       const double x2[3], const double v2[3], double R2, double *tc)
{
    double dx = x1[0] - x2[0], dy = x1[1] - x2[1], dz = x1[2] - x2[2];
    double ux = v1[0] - v2[0], uy = v1[1] - v2[1], uz = v1[2] - v2[2];
    double b = (dx * ux + dy * uy) + dz * uz;
    double dr2 = (dx * dx + dy * dy) + dz * dz;
    double dv2 = (ux * ux + uy * uy) + uz * uz;
    if (dv2 == 0.0) return 0;
    double Rs = R1 + R2;
    double Delta = b * b + dv2 * (Rs * Rs - dr2);
    if (Delta < 0.0) return 0;
    *tc = -(b + sqrt(Delta)) / dv2;
    return 1;
}

int or_collide_pair(const double x1[3], const double v1[3], double R1,
                    const double x2[3], const double v2[3], double R2, double dt)
{
    double tc;
    if (!impact_time(x1, v1, R1, x2, v2, R2, &tc)) return 0;
    return tc >= 0.0 && tc <= dt;
}

int64_t or_collide_brute(int64_t n, const double *pos, const double *vel, const double *R, double dt,
                         int64_t *pairs, int64_t cap)
{
    int64_t found = 0;
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = i + 1; j < n; j++)
            if (or_collide_pair(pos + 3 * i, vel + 3 * i, R[i], pos + 3 * j, vel + 3 * j, R[j], dt)) {
                if (found < cap) { pairs[2 * found] = i; pairs[2 * found + 1] = j; }
                found++;
            }
    return found;
}

/* ------------------------------------------------------------------------ */
/* Collision resolution (Sect. 5.1 and 5.2).  The two moonlets of a pair     */
/* (1, 2) = (i, j), i < j, move in straight lines to the impact at dt_c (the */
/* root of the predicate above), where, with dr = r1 - r2 and dv = v1 - v2   */
/* taken at the impact,                                                      */
/*   J = alpha (dr.dv) dr,  alpha = f m1 m2 / ((m1 + m2)(R1 + R2)^2),        */
/*   v1' = v1 - J / m1,     v2' = v2 + J / m2                                 */
/* (Eq. velocity_prediction; f = 2 is Eq. alpha_el, 1 <= f <= 2 Eq. alpha). */
/* The rest of the step is travelled at v': the position the drift starts    */
/* from becomes x + dt_c (v - v'), so that the drift x + dt v' lands on      */
/* (x + dt_c v) + (dt - dt_c) v' up to rounding.                             */
/* The paper does not say what happens to a moonlet found in several pairs   */
/* of one step.  Reading: pairs are taken in increasing (dt_c, i, j) and a   */
/* pair is resolved only if neither moonlet was resolved before it in the    */
/* step, so a moonlet has at most one impact per step, its earliest.         */
/* ------------------------------------------------------------------------ */
typedef struct { double tc; int64_t i, j, k; } Impact;

static int cmp_impact(const void *a, const void *b)
{
    const Impact *p = (const Impact *)a, *q = (const Impact *)b;
    if (p->tc != q->tc) return p->tc < q->tc ? -1 : 1;
    if (p->i != q->i) return p->i < q->i ? -1 : 1;
    if (p->j != q->j) return p->j < q->j ? -1 : 1;
    return 0;
}

static void resolve_pair(double *pos, double *vel, const double *mass, const double *rad, double f,
                         int64_t i, int64_t j, double tc)
{
    double *x1 = pos + 3 * i, *x2 = pos + 3 * j, *v1 = vel + 3 * i, *v2 = vel + 3 * j;
    double m1 = mass[i], m2 = mass[j];
    double Rs = rad[i] + rad[j];
    double dr[3], dv[3];
    for (int k = 0; k < 3; k++) {
        dr[k] = (x1[k] + tc * v1[k]) - (x2[k] + tc * v2[k]);
        dv[k] = v1[k] - v2[k];
    }
    double alpha = ((f * m1) * m2) / ((m1 + m2) * (Rs * Rs));
    double c = alpha * dot3(dr, dv);
    for (int k = 0; k < 3; k++) {
        double J = c * dr[k];
        double w1 = v1[k] - J / m1, w2 = v2[k] + J / m2;
        x1[k] = x1[k] + tc * (v1[k] - w1);
        x2[k] = x2[k] + tc * (v2[k] - w2);
        v1[k] = w1;
        v2[k] = w2;
    }
}

/* Resolves the colliding pairs (rows (i, j), i < j) of one step in place:  */
/* velocities become v', positions the drift's starting points.  done[k]    */
/* (nullable) tells whether pair k was resolved.  Returns how many were.    */
int64_t or_resolve(int64_t n, double *pos, double *vel, const double *mass, const double *rad, double f,
                   const int64_t *pairs, int64_t npairs, int64_t *done)
{
    Impact *im = (Impact *)malloc(sizeof(Impact) * (npairs > 0 ? npairs : 1));
    unsigned char *used = (unsigned char *)calloc(n > 0 ? n : 1, 1);
    int64_t m = 0, count = 0;
    for (int64_t k = 0; k < npairs; k++) {
        int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
        double tc;
        if (done) done[k] = 0;
        if (i < 0 || j >= n || i >= j) continue;
        if (!impact_time(pos + 3 * i, vel + 3 * i, rad[i], pos + 3 * j, vel + 3 * j, rad[j], &tc)) continue;
        im[m].tc = tc; im[m].i = i; im[m].j = j; im[m].k = k;
        m++;
    }
    qsort(im, (size_t)m, sizeof(Impact), cmp_impact);
    for (int64_t q = 0; q < m; q++) {
        if (used[im[q].i] || used[im[q].j]) continue;
        used[im[q].i] = used[im[q].j] = 1;
        resolve_pair(pos, vel, mass, rad, f, im[q].i, im[q].j, im[q].tc);
        if (done) done[im[q].k] = 1;
        count++;
    }
    free(im);
    free(used);
    return count;
}

/* ------------------------------------------------------------------------ */
/* Octree (Sect. 3.4.1).  Moonlets are taken in the order (Hilbert key,     */
/* index); a cell with more than s moonlets (and level < 21) is split into  */
/* the octants of its cube, given by the next bit of the quantised          */
/* coordinates; children are kept in order of first appearance.             */
/* ------------------------------------------------------------------------ */
typedef struct Node {
    int level;
    uint32_t c[3];          /* integer coordinates of the cell at its level */
    int64_t first, n;       /* members are ord[first .. first+n) */
    int nchild;
    struct Node *child[8];
    /* gravity climb */
    double M, s[3], rmax, rcrit;
    double *Mt, *Ct;        /* packed tensors */
    /* collision climb */
    double sb[3], rmax_c, rcrit_c;
} Node;

typedef struct {
    const or_params *P;
    int64_t n;
    const double *pos, *mass, *vel, *rad;
    double root[4];
    uint32_t *q;
    uint64_t *keys;
    int64_t *ord;           /* canonical order: user indices sorted by (key, index) */
    Node **nodes;
    int64_t nnodes, cap;
    Node *rootn;
    double Mtot;
    double *acc;            /* mutual acceleration, user order */
    double dt;
    int64_t *pairs, pcap, npairs;
    int64_t st[ST_NSTAT];
} Tree;

static const uint64_t *g_sort_keys;
static int cmp_key_idx(const void *a, const void *b)
{
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    if (g_sort_keys[i] < g_sort_keys[j]) return -1;
    if (g_sort_keys[i] > g_sort_keys[j]) return 1;
    return (i > j) - (i < j);
}

static Node *new_node(Tree *T, int level, const uint32_t c[3], int64_t first, int64_t n)
{
    Node *x = (Node *)calloc(1, sizeof(Node));
    x->level = level;
    x->c[0] = c[0]; x->c[1] = c[1]; x->c[2] = c[2];
    x->first = first;
    x->n = n;
    if (T->nnodes == T->cap) {
        T->cap = T->cap ? 2 * T->cap : 1024;
        T->nodes = (Node **)realloc(T->nodes, sizeof(Node *) * T->cap);
    }
    T->nodes[T->nnodes++] = x;
    return x;
}

static void split(Tree *T, Node *x)
{
    if (x->n <= T->P->leaf_size || x->level >= OR_BITS) return;
    int shift = OR_BITS - 1 - x->level;
    int64_t *buf = (int64_t *)malloc(sizeof(int64_t) * x->n);
    int64_t cnt[8] = {0};
    int order[8], norder = 0;
    for (int64_t k = 0; k < x->n; k++) {
        int64_t i = T->ord[x->first + k];
        int o = (int)((((T->q[3 * i] >> shift) & 1u) << 2) | (((T->q[3 * i + 1] >> shift) & 1u) << 1) |
                      ((T->q[3 * i + 2] >> shift) & 1u));
        if (cnt[o] == 0) order[norder++] = o;
        cnt[o]++;
    }
    int64_t start[8], at = x->first;
    for (int r = 0; r < norder; r++) { start[order[r]] = at; at += cnt[order[r]]; }
    int64_t fill[8];
    memcpy(fill, start, sizeof(fill));
    for (int64_t k = 0; k < x->n; k++) {
        int64_t i = T->ord[x->first + k];
        int o = (int)((((T->q[3 * i] >> shift) & 1u) << 2) | (((T->q[3 * i + 1] >> shift) & 1u) << 1) |
                      ((T->q[3 * i + 2] >> shift) & 1u));
        buf[fill[o]++ - x->first] = i;
    }
    memcpy(T->ord + x->first, buf, sizeof(int64_t) * x->n);
    free(buf);
    x->nchild = norder;
    for (int r = 0; r < norder; r++) {
        int o = order[r];
        uint32_t cc[3] = {(x->c[0] << 1) | ((o >> 2) & 1u), (x->c[1] << 1) | ((o >> 1) & 1u), (x->c[2] << 1) | (o & 1u)};
        x->child[r] = new_node(T, x->level + 1, cc, start[o], cnt[o]);
        split(T, x->child[r]);
    }
}

static void tree_build(Tree *T)
{
    int64_t n = T->n;
    T->q = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (n > 0 ? n : 1));
    T->keys = (uint64_t *)malloc(sizeof(uint64_t) * (n > 0 ? n : 1));
    T->ord = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    or_keys(n, T->pos, T->root, T->q, T->keys);
    for (int64_t i = 0; i < n; i++) T->ord[i] = i;
    g_sort_keys = T->keys;
    qsort(T->ord, (size_t)n, sizeof(int64_t), cmp_key_idx);
    uint32_t c0[3] = {0, 0, 0};
    T->rootn = new_node(T, 0, c0, 0, n);
    split(T, T->rootn);
}

static void tree_free(Tree *T)
{
    for (int64_t k = 0; k < T->nnodes; k++) {
        free(T->nodes[k]->Mt);
        free(T->nodes[k]->Ct);
        free(T->nodes[k]);
    }
    free(T->nodes);
    free(T->q);
    free(T->keys);
    free(T->ord);
}

/* distance from s to the farthest corner of the cell's cube, the cube being
 * widened by L 2^-48 on every side so that rounding in the quantisation can
 * never leave a member outside it (corner cap of Sect. 3.4.2) */
static double corner_distance(const Tree *T, const Node *x, const double s[3])
{
    double L = T->root[3];
    double h = L;
    for (int k = 0; k < x->level; k++) h *= 0.5;
    double eps = L * 0x1p-48;
    double acc = 0.0;
    double d[3];
    for (int k = 0; k < 3; k++) {
        double lo = T->root[k] + (double)x->c[k] * h;
        double a = s[k] - (lo - eps), b = ((lo + h) + eps) - s[k];
        d[k] = a > b ? a : b;
    }
    acc = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
    return sqrt(acc);
}

/* ---- gravity climb (Eqs. expansion_center, rmax_2, rcrit_2; corner cap) ---- */
static void climb_gravity(Tree *T, Node *x)
{
    const or_params *P = T->P;
    double sx = 0.0, sy = 0.0, sz = 0.0, M = 0.0;
    if (x->nchild == 0) {
        for (int64_t k = 0; k < x->n; k++) {
            int64_t i = T->ord[x->first + k];
            double m = T->mass[i];
            M = M + m;
            sx = sx + m * T->pos[3 * i];
            sy = sy + m * T->pos[3 * i + 1];
            sz = sz + m * T->pos[3 * i + 2];
        }
        x->M = M;
        x->s[0] = sx / M; x->s[1] = sy / M; x->s[2] = sz / M;
        double rmax = 0.0;
        for (int64_t k = 0; k < x->n; k++) {
            int64_t i = T->ord[x->first + k];
            double d[3] = {T->pos[3 * i] - x->s[0], T->pos[3 * i + 1] - x->s[1], T->pos[3 * i + 2] - x->s[2]};
            double r = norm3(d);
            if (r > rmax) rmax = r;
        }
        x->rmax = rmax;
    } else {
        for (int c = 0; c < x->nchild; c++) climb_gravity(T, x->child[c]);
        for (int c = 0; c < x->nchild; c++) {
            Node *y = x->child[c];
            M = M + y->M;
            sx = sx + y->M * y->s[0];
            sy = sy + y->M * y->s[1];
            sz = sz + y->M * y->s[2];
        }
        x->M = M;
        x->s[0] = sx / M; x->s[1] = sy / M; x->s[2] = sz / M;
        double rmax = 0.0;
        for (int c = 0; c < x->nchild; c++) {
            Node *y = x->child[c];
            double d[3] = {y->s[0] - x->s[0], y->s[1] - x->s[1], y->s[2] - x->s[2]};
            double r = y->rmax + norm3(d);
            if (r > rmax) rmax = r;
        }
        x->rmax = rmax;
    }
    double cap = corner_distance(T, x, x->s);
    if (cap < x->rmax) x->rmax = cap;
    /* multipoles (Eq. multipole_moment at leaves, App. C at parents) */
    int tot = OFF(P->p);
    x->Mt = (double *)calloc((size_t)tot, sizeof(double));
    if (x->nchild == 0 || P->m2m_direct) {
        double tmp[729];
        for (int64_t k = 0; k < x->n; k++) {
            int64_t i = T->ord[x->first + k];
            double mu = P->G * T->mass[i];
            double d[3] = {T->pos[3 * i] - x->s[0], T->pos[3 * i + 1] - x->s[1], T->pos[3 * i + 2] - x->s[2]};
            for (int nn = 0; nn < P->p; nn++) {
                if (nn == 1) continue;
                outer_power(d, nn, tmp);
                for (int t = 0; t < POW3[nn]; t++) x->Mt[OFF(nn) + t] += mu * tmp[t];
            }
        }
    } else {
        for (int c = 0; c < x->nchild; c++) or_m2m(P->p, x->child[c]->Mt, x->child[c]->s, x->s, x->Mt);
        for (int t = 0; t < 3 && P->p > 1; t++) x->Mt[OFF(1) + t] = 0.0;
    }
}

static void finish_gravity(Tree *T)
{
    T->Mtot = T->rootn->M;
    for (int64_t k = 0; k < T->nnodes; k++) {
        Node *x = T->nodes[k];
        x->rcrit = x->rmax / or_theta(x->M, T->Mtot, T->P->theta_min);
        x->Ct = (double *)calloc((size_t)OFF(T->P->p + 1), sizeof(double));
    }
}

/* ---- collision climb (Eqs. center, rmax, rcrit; corner cap) ----
 * Eq. center is read as the mean position of the moonlets contained: at a
 * parent each child's mean is weighted by its number of moonlets. */
static void climb_collision(Tree *T, Node *x)
{
    double dt = T->dt;
    double sx = 0.0, sy = 0.0, sz = 0.0, ex = 0.0;
    if (x->nchild == 0) {
        for (int64_t k = 0; k < x->n; k++) {
            int64_t i = T->ord[x->first + k];
            sx = sx + T->pos[3 * i];
            sy = sy + T->pos[3 * i + 1];
            sz = sz + T->pos[3 * i + 2];
        }
        double cnt = (double)x->n;
        x->sb[0] = sx / cnt; x->sb[1] = sy / cnt; x->sb[2] = sz / cnt;
        double rmax = 0.0;
        for (int64_t k = 0; k < x->n; k++) {
            int64_t i = T->ord[x->first + k];
            double d[3] = {T->pos[3 * i] - x->sb[0], T->pos[3 * i + 1] - x->sb[1], T->pos[3 * i + 2] - x->sb[2]};
            double r = norm3(d);
            if (r > rmax) rmax = r;
            double e = T->rad[i] + dt * norm3(T->vel + 3 * i);   /* r_crit,a - r_max,a of a moonlet */
            if (e > ex) ex = e;
        }
        x->rmax_c = rmax;
    } else {
        for (int c = 0; c < x->nchild; c++) climb_collision(T, x->child[c]);
        for (int c = 0; c < x->nchild; c++) {
            Node *y = x->child[c];
            double w = (double)y->n;
            sx = sx + w * y->sb[0];
            sy = sy + w * y->sb[1];
            sz = sz + w * y->sb[2];
        }
        double cnt = (double)x->n;
        x->sb[0] = sx / cnt; x->sb[1] = sy / cnt; x->sb[2] = sz / cnt;
        double rmax = 0.0;
        for (int c = 0; c < x->nchild; c++) {
            Node *y = x->child[c];
            double d[3] = {y->sb[0] - x->sb[0], y->sb[1] - x->sb[1], y->sb[2] - x->sb[2]};
            double r = y->rmax_c + norm3(d);
            if (r > rmax) rmax = r;
            double e = y->rcrit_c - y->rmax_c;
            if (e > ex) ex = e;
        }
        x->rmax_c = rmax;
    }
    double cap = corner_distance(T, x, x->sb);
    if (cap < x->rmax_c) x->rmax_c = cap;
    x->rcrit_c = x->rmax_c + ex;
}

/* ------------------------------------------------------------------------ */
/* Interactions.                                                            */
/* ------------------------------------------------------------------------ */
static void p2p_pair(Tree *T, int64_t i, int64_t j)
{
    const double *xi = T->pos + 3 * i, *xj = T->pos + 3 * j;
    double d[3] = {xi[0] - xj[0], xi[1] - xj[1], xi[2] - xj[2]};
    double r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
    T->st[ST_P2P_INTER]++;
    if (r2 == 0.0) return;
    double r = sqrt(r2);
    double inv3 = 1.0 / (r2 * r);
    double fi = T->P->G * T->mass[j] * inv3, fj = T->P->G * T->mass[i] * inv3;
    for (int k = 0; k < 3; k++) {
        T->acc[3 * i + k] -= fi * d[k];
        T->acc[3 * j + k] += fj * d[k];
    }
}

static void col_pair(Tree *T, int64_t i, int64_t j)
{
    int64_t a = i < j ? i : j, b = i < j ? j : i;
    T->st[ST_COL_TESTS]++;
    if (or_collide_pair(T->pos + 3 * a, T->vel + 3 * a, T->rad[a], T->pos + 3 * b, T->vel + 3 * b, T->rad[b], T->dt)) {
        if (T->npairs < T->pcap) { T->pairs[2 * T->npairs] = a; T->pairs[2 * T->npairs + 1] = b; }
        T->npairs++;
    }
}

static void direct_self(Tree *T, Node *A, int gravity)
{
    for (int64_t u = 0; u < A->n; u++)
        for (int64_t v = u + 1; v < A->n; v++) {
            int64_t i = T->ord[A->first + u], j = T->ord[A->first + v];
            if (gravity) p2p_pair(T, i, j); else col_pair(T, i, j);
        }
}

static void direct_pair(Tree *T, Node *A, Node *B, int gravity)
{
    for (int64_t u = 0; u < A->n; u++)
        for (int64_t v = 0; v < B->n; v++) {
            int64_t i = T->ord[A->first + u], j = T->ord[B->first + v];
            if (gravity) p2p_pair(T, i, j); else col_pair(T, i, j);
        }
}

/* ---- Algorithm TreeWalk (Sect. 3.4.5).
 * What happens to a pending pair of cells (A, B) is one decision, made by
 * walk_choice() from the pair alone; the walk itself keeps the pending pairs
 * on an explicit stack, starting from (root, root).  Children replace their
 * parent pair in the order the algorithm visits them (pushed in reverse, so
 * they are taken in order), which gives the same sequence of interactions
 * as a depth-first recursion.
 * gravity = 1: M2L for well-separated pairs; gravity = 0: collision search,
 * where well-separated pairs are pruned (with a relative margin 2^-40) and
 * every "brute force" outcome tests the moonlet pairs. */
typedef enum {
    WALK_SELF_DIRECT,   /* A == B, few moonlets or a leaf: all pairs inside A */
    WALK_SELF_OPEN,     /* A == B: every pair (a, b), a <= b, of children */
    WALK_DIRECT,        /* all pairs of A x B */
    WALK_FAR,           /* well separated: M2L (gravity) or nothing (collisions) */
    WALK_OPEN_A,        /* (a, B) for every child a of A */
    WALK_OPEN_B         /* (A, b) for every child b of B */
} WalkChoice;

static int well_separated(const Node *A, const Node *B, int gravity)
{
    if (gravity) {   /* (r_crit,A + r_crit,B)^2 <= |s_A - s_B|^2 */
        double d[3] = {A->s[0] - B->s[0], A->s[1] - B->s[1], A->s[2] - B->s[2]};
        double d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
        double t = A->rcrit + B->rcrit;
        return t * t <= d2;
    }
    double d[3] = {A->sb[0] - B->sb[0], A->sb[1] - B->sb[1], A->sb[2] - B->sb[2]};
    double d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
    double t = (A->rcrit_c + B->rcrit_c) * (1.0 + 0x1p-40);
    return t * t < d2;
}

static WalkChoice walk_choice(const or_params *P, const Node *A, const Node *B, int gravity)
{
    int64_t n_cs = gravity ? P->n_cs : P->c_cs;
    int64_t n_pre = gravity ? P->n_cc_pre : P->c_cc_pre;
    int64_t n_post = gravity ? P->n_cc_post : P->c_cc_post;
    int leafA = A->nchild == 0, leafB = B->nchild == 0;
    if (A == B) return (A->n <= n_cs || leafA) ? WALK_SELF_DIRECT : WALK_SELF_OPEN;
    int64_t prod = A->n * B->n;
    if (prod < n_pre) return WALK_DIRECT;
    if (well_separated(A, B, gravity)) return WALK_FAR;
    if (prod < n_post || (leafA && leafB)) return WALK_DIRECT;
    /* split the larger (by r_crit) of the two, never a leaf (reading c5) */
    double rA = gravity ? A->rcrit : A->rcrit_c, rB = gravity ? B->rcrit : B->rcrit_c;
    return (!leafA && (rA > rB || leafB)) ? WALK_OPEN_A : WALK_OPEN_B;
}

typedef struct { Node **a, **b; int64_t top, cap; } PairStack;

static void push_pair(PairStack *S, Node *a, Node *b)
{
    if (S->top == S->cap) {
        S->cap = S->cap ? 2 * S->cap : 256;
        S->a = (Node **)realloc(S->a, sizeof(Node *) * S->cap);
        S->b = (Node **)realloc(S->b, sizeof(Node *) * S->cap);
    }
    S->a[S->top] = a;
    S->b[S->top] = b;
    S->top++;
}

static void tree_walk(Tree *T, Node *root, int gravity)
{
    PairStack S = {NULL, NULL, 0, 0};
    push_pair(&S, root, root);
    while (S.top > 0) {
        S.top--;
        Node *A = S.a[S.top], *B = S.b[S.top];
        switch (walk_choice(T->P, A, B, gravity)) {
        case WALK_SELF_DIRECT:
            T->st[gravity ? ST_P2P_SELF : ST_COL_SELF]++;
            direct_self(T, A, gravity);
            break;
        case WALK_SELF_OPEN:   /* visited in the order (0,0), (0,1), ..., (1,1), ... */
            for (int a = A->nchild - 1; a >= 0; a--)
                for (int b = A->nchild - 1; b >= a; b--) push_pair(&S, A->child[a], A->child[b]);
            break;
        case WALK_DIRECT:
            T->st[gravity ? ST_P2P_PAIRS : ST_COL_PAIRS]++;
            direct_pair(T, A, B, gravity);
            break;
        case WALK_FAR:
            if (gravity) {
                T->st[ST_M2L]++;
                or_m2l(T->P->p, A->s, A->Mt, B->s, B->Mt, A->Ct, B->Ct);
            }
            break;
        case WALK_OPEN_A:
            for (int a = A->nchild - 1; a >= 0; a--) push_pair(&S, A->child[a], B);
            break;
        case WALK_OPEN_B:
            for (int b = B->nchild - 1; b >= 0; b--) push_pair(&S, A, B->child[b]);
            break;
        }
    }
    free(S.a);
    free(S.b);
}

/* ---- Algorithm StandardTree (Sect. 3.4.4), gravity, for moonlet a and cell
 * B: brute force when B holds fewer than N_cb,pre moonlets; the expansion of
 * B at a (M2P) when a is well separated from B; brute force when B holds
 * fewer than N_cb,post moonlets or is a leaf; else the children of B in
 * turn.  A moonlet is a point (r_crit = 0), so "well separated" reads
 * r_crit,B^2 <= |x_a - s_B|^2, in FP64 in a fixed order; a moonlet at the
 * centre itself (a one-moonlet cell, r_crit = 0, seen from its own moonlet)
 * is not, since the expansion is singular there.  Brute force adds the pull
 * of every moonlet of B on a alone (coincident moonlets, a itself included,
 * are skipped). */
static void direct_one(Tree *T, int64_t a, Node *B)
{
    const double *xa = T->pos + 3 * a;
    T->st[ST_P2P_PAIRS]++;
    for (int64_t v = 0; v < B->n; v++) {
        int64_t j = T->ord[B->first + v];
        const double *xj = T->pos + 3 * j;
        double d[3] = {xa[0] - xj[0], xa[1] - xj[1], xa[2] - xj[2]};
        double r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
        T->st[ST_P2P_INTER]++;
        if (r2 == 0.0) continue;
        double r = sqrt(r2);
        double f = T->P->G * T->mass[j] * (1.0 / (r2 * r));
        for (int k = 0; k < 3; k++) T->acc[3 * a + k] -= f * d[k];
    }
}

static void standard_tree(Tree *T, int64_t a, Node *B)
{
    const or_params *P = T->P;
    if (B->n < P->n_cb_pre) { direct_one(T, a, B); return; }
    const double *xa = T->pos + 3 * a;
    double d[3] = {xa[0] - B->s[0], xa[1] - B->s[1], xa[2] - B->s[2]};
    double d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
    if (d2 > 0.0 && B->rcrit * B->rcrit <= d2) {
        T->st[ST_M2L]++;
        or_m2p(P->p, xa, B->s, B->Mt, T->acc + 3 * a);
        return;
    }
    if (B->n < P->n_cb_post || B->nchild == 0) { direct_one(T, a, B); return; }
    for (int c = 0; c < B->nchild; c++) standard_tree(T, a, B->child[c]);
}

/* ---- Algorithm StandardTree for collision search (Sect. 3.4.4, the
 * instructions for collisions): brute force when B holds fewer than
 * N_cb,pre moonlets; nothing when a is well separated from B; brute force
 * when B holds fewer than N_cb,post moonlets or is a leaf; else the children.
 * The moonlet's r_crit is R_a + dt |v_a| (r_max = 0, Eq. rcrit) and pruning
 * keeps the relative margin of the dual walk:
 * ((r_crit,a + r_crit,B)(1 + 2^-40))^2 < |x_a - sbar_B|^2.  Brute force
 * tests a against the moonlets of B with a larger caller index, so each
 * pair is tested from the walk of its lower index (which reaches it: only
 * pairs that cannot touch are pruned). */
static void col_one(Tree *T, int64_t a, Node *B)
{
    T->st[ST_COL_PAIRS]++;
    for (int64_t v = 0; v < B->n; v++) {
        int64_t j = T->ord[B->first + v];
        if (j > a) col_pair(T, a, j);
    }
}

static void standard_collide(Tree *T, int64_t a, Node *B, double rca)
{
    const or_params *P = T->P;
    if (B->n < P->c_cb_pre) { col_one(T, a, B); return; }
    const double *xa = T->pos + 3 * a;
    double d[3] = {xa[0] - B->sb[0], xa[1] - B->sb[1], xa[2] - B->sb[2]};
    double d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
    double t = (rca + B->rcrit_c) * (1.0 + 0x1p-40);
    if (t * t < d2) return;
    if (B->n < P->c_cb_post || B->nchild == 0) { col_one(T, a, B); return; }
    for (int c = 0; c < B->nchild; c++) standard_collide(T, a, B->child[c], rca);
}

/* ---- tree descent: L2L from the root, L2P at the leaves (Eq. shifting) */
static void descend(Tree *T, Node *x)
{
    int p = T->P->p;
    if (x->nchild == 0) {
        for (int64_t k = 0; k < x->n; k++) {
            int64_t i = T->ord[x->first + k];
            or_l2p(p, x->Ct, x->s, T->pos + 3 * i, T->acc + 3 * i);
        }
        return;
    }
    for (int c = 0; c < x->nchild; c++) {
        or_l2l(p, x->Ct, x->s, x->child[c]->s, x->child[c]->Ct);
        descend(T, x->child[c]);
    }
}

static int cmp_node(const void *a, const void *b)
{
    const Node *x = *(Node *const *)a, *y = *(Node *const *)b;
    if (x->level != y->level) return x->level - y->level;
    return (x->first > y->first) - (x->first < y->first);
}

static void tree_stats(Tree *T)
{
    T->st[ST_CELLS] = T->nnodes;
    int64_t leaves = 0, depth = 0;
    for (int64_t k = 0; k < T->nnodes; k++) {
        if (T->nodes[k]->nchild == 0) leaves++;
        if (T->nodes[k]->level > depth) depth = T->nodes[k]->level;
    }
    T->st[ST_LEAVES] = leaves;
    T->st[ST_DEPTH] = depth;
}

/* ------------------------------------------------------------------------ */
/* Exported drivers.                                                        */
/* ------------------------------------------------------------------------ */

/* falcON mutual acceleration (without external forces), user order. */
int or_falcon_accel(const or_params *P, int64_t n, const double *pos, const double *mass,
                    double *acc, int64_t *stats)
{
    Tree T;
    memset(&T, 0, sizeof(T));
    T.P = P; T.n = n; T.pos = pos; T.mass = mass; T.acc = acc;
    memset(acc, 0, sizeof(double) * 3 * (n > 0 ? n : 0));
    if (n <= 0) return 0;
    tree_build(&T);
    climb_gravity(&T, T.rootn);
    finish_gravity(&T);
    tree_walk(&T, T.rootn, 1);
    descend(&T, T.rootn);
    tree_stats(&T);
    if (stats) memcpy(stats, T.st, sizeof(T.st));
    tree_free(&T);
    return 0;
}

/* Standard tree code mutual acceleration (Algorithm StandardTree called with
 * (moonlet a, root) for every moonlet), user order, no external forces.
 * Stats: ST_M2L counts moonlet-cell expansions (M2P), ST_P2P_PAIRS the
 * brute-force moonlet-cell interactions, ST_P2P_INTER their moonlet pairs. */
int or_standard_accel(const or_params *P, int64_t n, const double *pos, const double *mass,
                      double *acc, int64_t *stats)
{
    Tree T;
    memset(&T, 0, sizeof(T));
    T.P = P; T.n = n; T.pos = pos; T.mass = mass; T.acc = acc;
    memset(acc, 0, sizeof(double) * 3 * (n > 0 ? n : 0));
    if (n <= 0) return 0;
    tree_build(&T);
    climb_gravity(&T, T.rootn);
    finish_gravity(&T);
    for (int64_t a = 0; a < n; a++) standard_tree(&T, a, T.rootn);
    tree_stats(&T);
    if (stats) memcpy(stats, T.st, sizeof(T.st));
    tree_free(&T);
    return 0;
}

/* Per-cell expansions for parity of the multipole stages: after the climb,
 * the walk and the descent, cells in level-major order; M: packed full tensors
 * of orders 0..p-1 (OFF(p) values per cell), C: the complete local expansion
 * of each cell (its M2L sums plus its ancestors' translated to its centre),
 * orders 0..p (OFF(p+1) values per cell, order 0 unused).  Returns the cell
 * count. */
int64_t or_expansions(const or_params *P, int64_t n, const double *pos, const double *mass,
                      double *Mout, double *Cout, int64_t cap)
{
    if (n <= 0) return 0;
    Tree T;
    memset(&T, 0, sizeof(T));
    T.P = P; T.n = n; T.pos = pos; T.mass = mass;
    T.acc = (double *)calloc((size_t)3 * n, sizeof(double));
    tree_build(&T);
    climb_gravity(&T, T.rootn);
    finish_gravity(&T);
    tree_walk(&T, T.rootn, 1);
    descend(&T, T.rootn);
    Node **sorted = (Node **)malloc(sizeof(Node *) * T.nnodes);
    memcpy(sorted, T.nodes, sizeof(Node *) * T.nnodes);
    qsort(sorted, (size_t)T.nnodes, sizeof(Node *), cmp_node);
    int nm = OFF(P->p), nc = OFF(P->p + 1);
    for (int64_t k = 0; k < T.nnodes && k < cap; k++) {
        if (Mout) memcpy(Mout + (size_t)k * nm, sorted[k]->Mt, sizeof(double) * nm);
        if (Cout) memcpy(Cout + (size_t)k * nc, sorted[k]->Ct, sizeof(double) * nc);
    }
    int64_t cnt = T.nnodes;
    free(sorted);
    free(T.acc);
    tree_free(&T);
    return cnt;
}

/* tree-based collision search (pairs user indices, sorted, i < j) */
static int cmp_pair(const void *a, const void *b)
{
    const int64_t *x = (const int64_t *)a, *y = (const int64_t *)b;
    if (x[0] != y[0]) return (x[0] > y[0]) - (x[0] < y[0]);
    return (x[1] > y[1]) - (x[1] < y[1]);
}

int64_t or_collide_tree(const or_params *P, int64_t n, const double *pos, const double *vel,
                        const double *rad, double dt, int64_t *pairs, int64_t cap, int64_t *stats)
{
    if (n <= 0) return 0;
    Tree T;
    memset(&T, 0, sizeof(T));
    T.P = P; T.n = n; T.pos = pos; T.vel = vel; T.rad = rad; T.dt = dt;
    T.pairs = pairs; T.pcap = cap;
    tree_build(&T);
    climb_collision(&T, T.rootn);
    tree_walk(&T, T.rootn, 0);
    int64_t found = T.npairs;
    if (found <= cap) qsort(pairs, (size_t)found, 2 * sizeof(int64_t), cmp_pair);
    tree_stats(&T);
    T.st[ST_COL_FOUND] = found;
    if (stats) memcpy(stats, T.st, sizeof(T.st));
    tree_free(&T);
    return found;
}

/* Collision search by the standard tree code (Algorithm StandardTree called
 * with (moonlet a, root) for every moonlet); pairs in user indices, i < j,
 * sorted when they fit.  Stats: ST_COL_PAIRS = brute-force moonlet-cell
 * interactions, ST_COL_TESTS = pairs tested, ST_COL_FOUND. */
int64_t or_collide_standard(const or_params *P, int64_t n, const double *pos, const double *vel,
                            const double *rad, double dt, int64_t *pairs, int64_t cap, int64_t *stats)
{
    if (n <= 0) return 0;
    Tree T;
    memset(&T, 0, sizeof(T));
    T.P = P; T.n = n; T.pos = pos; T.vel = vel; T.rad = rad; T.dt = dt;
    T.pairs = pairs; T.pcap = cap;
    tree_build(&T);
    climb_collision(&T, T.rootn);
    for (int64_t a = 0; a < n; a++)
        standard_collide(&T, a, T.rootn, rad[a] + dt * norm3(vel + 3 * a));
    int64_t found = T.npairs;
    if (found <= cap) qsort(pairs, (size_t)found, 2 * sizeof(int64_t), cmp_pair);
    tree_stats(&T);
    T.st[ST_COL_FOUND] = found;
    if (stats) memcpy(stats, T.st, sizeof(T.st));
    tree_free(&T);
    return found;
}

/* Tree export for parity: canonical order, keys, and per cell (level-major,
 * then by first member): level, cx, cy, cz, first, count, nchild as int64
 * rows of 7, plus gravity geometry (M, sx, sy, sz, rmax, rcrit) and collision
 * geometry (sbx, sby, sbz, rmax_c, rcrit_c) when the matching input is
 * given.  Returns the number of cells (rows beyond cap are not written). */
int64_t or_tree_export(const or_params *P, int64_t n, const double *pos, const double *mass,
                       const double *vel, const double *rad, double dt,
                       int64_t *ord, uint64_t *keys, double *root,
                       int64_t *cells, double *ggeo, double *cgeo, int64_t cap)
{
    if (n <= 0) return 0;
    Tree T;
    memset(&T, 0, sizeof(T));
    T.P = P; T.n = n; T.pos = pos; T.mass = mass; T.vel = vel; T.rad = rad; T.dt = dt;
    tree_build(&T);
    if (mass) { climb_gravity(&T, T.rootn); finish_gravity(&T); }
    if (vel && rad) climb_collision(&T, T.rootn);
    if (ord) memcpy(ord, T.ord, sizeof(int64_t) * n);
    if (keys) memcpy(keys, T.keys, sizeof(uint64_t) * n);
    if (root) memcpy(root, T.root, sizeof(double) * 4);
    Node **sorted = (Node **)malloc(sizeof(Node *) * T.nnodes);
    memcpy(sorted, T.nodes, sizeof(Node *) * T.nnodes);
    qsort(sorted, (size_t)T.nnodes, sizeof(Node *), cmp_node);
    for (int64_t k = 0; k < T.nnodes && k < cap; k++) {
        Node *x = sorted[k];
        if (cells) {
            int64_t *r = cells + 7 * k;
            r[0] = x->level; r[1] = x->c[0]; r[2] = x->c[1]; r[3] = x->c[2];
            r[4] = x->first; r[5] = x->n; r[6] = x->nchild;
        }
        if (ggeo && mass) {
            double *g = ggeo + 6 * k;
            g[0] = x->M; g[1] = x->s[0]; g[2] = x->s[1]; g[3] = x->s[2]; g[4] = x->rmax; g[5] = x->rcrit;
        }
        if (cgeo && vel && rad) {
            double *g = cgeo + 5 * k;
            g[0] = x->sb[0]; g[1] = x->sb[1]; g[2] = x->sb[2]; g[3] = x->rmax_c; g[4] = x->rcrit_c;
        }
    }
    int64_t cnt = T.nnodes;
    free(sorted);
    tree_free(&T);
    return cnt;
}

/* ---- SBAB1 kick-drift-kick with merged kicks (Sect. 4.1).
 * acc0: acceleration at the input positions (mutual + external), or NULL to
 * compute it.  Each step: v += dt/2 a; search collisions on (x, v); x += dt v;
 * a = falcON + external at the new x and time t + dt; v += dt/2 a.
 * With P->resolve_f > 0 the pairs are resolved (or_resolve) between the
 * search and the drift.  Collision pairs of step k are stored with a leading
 * step index: rows (k, i, j).  The final acceleration is left in acc_out;
 * *resolved (nullable) receives the number of resolved impacts, or -1 when
 * a step found more pairs than cap (then nothing more is resolved). */
int64_t or_kdk(const or_params *P0, int64_t n, double *pos, double *vel, const double *mass,
               const double *rad, double dt, int nsteps, const double *acc0, double *acc_out,
               int64_t *pairs, int64_t cap, int64_t *resolved)
{
    or_params P = *P0;
    double *a = (double *)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * 2 * (cap > 0 ? cap : 1));
    int64_t total = 0, nres = 0;
    if (acc0) memcpy(a, acc0, sizeof(double) * 3 * n);
    else {
        or_falcon_accel(&P, n, pos, mass, a, NULL);
        or_external_accel(&P, n, pos, P.time, a);
    }
    double h = 0.5 * dt;
    for (int s = 0; s < nsteps; s++) {
        for (int64_t i = 0; i < 3 * n; i++) vel[i] = vel[i] + h * a[i];
        int64_t found = P.brute_collisions ? or_collide_brute(n, pos, vel, rad, dt, tmp, cap)
                                           : or_collide_tree(&P, n, pos, vel, rad, dt, tmp, cap, NULL);
        for (int64_t k = 0; k < found; k++) {
            if (total < cap) {
                pairs[3 * total] = s; pairs[3 * total + 1] = tmp[2 * k]; pairs[3 * total + 2] = tmp[2 * k + 1];
            }
            total++;
        }
        if (P.resolve_f > 0.0 && nres >= 0) {
            if (found > cap) nres = -1;
            else nres += or_resolve(n, pos, vel, mass, rad, P.resolve_f, tmp, found, NULL);
        }
        for (int64_t i = 0; i < 3 * n; i++) pos[i] = pos[i] + dt * vel[i];
        P.time = P.time + dt;
        or_falcon_accel(&P, n, pos, mass, a, NULL);
        or_external_accel(&P, n, pos, P.time, a);
        for (int64_t i = 0; i < 3 * n; i++) vel[i] = vel[i] + h * a[i];
    }
    if (acc_out) memcpy(acc_out, a, sizeof(double) * 3 * n);
    if (resolved) *resolved = nres;
    free(a);
    free(tmp);
    return total;
}
