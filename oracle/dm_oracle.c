/*
 * CPU oracle for the discrete-continuous dense stereo method of
 * Shekhovtsov, Reinbacher, Graber, Pock, "Solving Dense Image Matching in
 * Real-Time using Discrete-Continuous Optimization" (arXiv 1601.06274).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  The product (the CUDA
 * library) never links, calls or reads anything in this directory, and this
 * file shares no code, header, table or constant with it.
 *
 * The oracle is deliberately plain and slow:
 *   - the discrete stage runs in int64 with O(K^2) explicit message
 *     minimisation and the hierarchical minorant as a plain recursion that
 *     recomputes every message it needs (no reuse, no normalisation);
 *   - the continuous stage runs in double precision, one formula per line.
 *
 * Readings of points the paper leaves open (each is also listed with its
 * justification in the design notes of the repository):
 *   R1  census window w x w (default 5), bit = [I(neighbour) < I(centre)],
 *       clamp-to-edge borders;  cost = popcount(cL(x) ^ cR(x - l)), and
 *       w*w - 1 when x - l < 0.
 *   R2  label l <-> disparity l pixels.
 *   R3  edge weight omega = w_hi if |I1(i) - I1(j)| < T else w_lo.
 *   R4  the discrete pairwise term is omega * r(|x_i - x_j|) with r of Eq.
 *       (r-decompose) sampled at integers (must be integer valued).
 *   R5  Dual MM starts from the zero minorant of the vertical chains, puts the
 *       whole data cost in the horizontal chains, and one iteration is a
 *       horizontal pass followed by a vertical pass.
 *   R6  hierarchical minorant: left part of a split has ceil(n/2) nodes; the
 *       "half" of the min-marginal in the Handshake is floor(m/2) (toward
 *       minus infinity); singletons take their whole min-marginal.
 *   R7  output labelling = per-pixel argmin of lam_h + lam_v (ties -> the
 *       smallest label); lower bound = sum_i min_l (lam_h + lam_v)_i(l).
 *   R8  continuous data term D_i = piecewise-linear interpolation of the
 *       cost samples, with the argument clamped to [0, L-1].
 *   R9  linearisation slopes s1 = (D(u0) - D(u0-h))/h (left),
 *       s2 = (D(u0+h) - D(u0))/h (right), both := mean if s2 < s1;
 *       box [u0-h, u0+h] intersected with [0, L-1].
 *   R10 data prox middle case returns u0 (the kink), then clamps to the box.
 *   R11 conjugate (omega r_{a,b})*(s) = b * max(0, |s| - omega a) for
 *       |s| <= omega, +inf otherwise; prox of Eq. (pprox) with step sigma.
 *   R12 u0 = labels, p = q = 0; the (u, q) step uses the old (u, p, q); the
 *       p step uses the extrapolation 2u+ - u; iterations are split evenly over
 *       the warps (earlier warps take the remainder).
 */

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef int64_t i64;

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_NONINTEGER 2

/* ------------------------------------------------------------------------ */
/* Census transform and matching cost (Sec. 3.1: census on a small patch,    */
/* pixel-wise Hamming distance; Sec. 1: the cost is precomputed for every     */
/* label).                                                                    */
/* ------------------------------------------------------------------------ */

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* census bit k (k = 0, 1, ...) is the k-th window neighbour in raster order,
 * centre skipped: bit = I(neighbour) < I(centre) (reading R1) */
int or_census(int H, int W, const uint8_t* img, int win, uint32_t* out)
{
    if (H <= 0 || W <= 0 || (win != 3 && win != 5)) return OR_ERR_ARG;
    int r = win / 2;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            uint32_t code = 0;
            int bit = 0;
            int centre = img[y * W + x];
            for (int dy = -r; dy <= r; ++dy)
                for (int dx = -r; dx <= r; ++dx) {
                    if (dy == 0 && dx == 0) continue;
                    int yy = clampi(y + dy, 0, H - 1), xx = clampi(x + dx, 0, W - 1);
                    if (img[yy * W + xx] < centre) code |= (1u << bit);
                    ++bit;
                }
            out[y * W + x] = code;
        }
    return OR_OK;
}

static int popcount32(uint32_t v)
{
    int c = 0;
    while (v) { c += (int)(v & 1u); v >>= 1; }
    return c;
}

/* c[y][x][l] = Hamming(cL[y][x], cR[y][x-l]), or maxc if x - l < 0 (R1, R2) */
int or_cost_volume(int H, int W, int L, const uint32_t* cl, const uint32_t* cr, int maxc,
                   int32_t* cost)
{
    if (H <= 0 || W <= 0 || L <= 0) return OR_ERR_ARG;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int l = 0; l < L; ++l) {
                int32_t v = maxc;
                if (x - l >= 0) v = popcount32(cl[y * W + x] ^ cr[y * W + x - l]);
                cost[((i64)y * W + x) * L + l] = v;
            }
    return OR_OK;
}

/* Right-view matching cost for the two-sided consistency check (Sec. 4.1.1
 * names the check, the caption of Table 1 its doubled cost; reading R25): the
 * right image is the reference, and its pixel x under label l is matched with
 * the left image's pixel x + l:
 * c[y][x][l] = Hamming(cR[y][x], cL[y][x+l]), or maxc if x + l >= W. */
int or_cost_volume_right(int H, int W, int L, const uint32_t* cl, const uint32_t* cr, int maxc,
                         int32_t* cost)
{
    if (H <= 0 || W <= 0 || L <= 0) return OR_ERR_ARG;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int l = 0; l < L; ++l) {
                int32_t v = maxc;
                if (x + l < W) v = popcount32(cr[y * W + x] ^ cl[y * W + x + l]);
                cost[((i64)y * W + x) * L + l] = v;
            }
    return OR_OK;
}

/* Two-sided consistency check (Sec. 4.1.1: the outliers that the truncated
 * regulariser lets through are removed by checking the two views against each
 * other; readings R26-R28).  The left pixel (y, x) with disparity d = ul[y][x]
 * has its counterpart in the right view at xr = x - rint(d) (nearest integer,
 * ties to even).  It passes when 0 <= xr < W and |d - ur[y][xr]| <= max_diff,
 * the difference taken in single precision, the precision of the disparities.
 * ok = 1 where it passes, else 0; out = d where it passes, else -1. */
int or_lr_check(int H, int W, const float* ul, const float* ur, float max_diff, uint8_t* ok,
                float* out)
{
    if (H <= 0 || W <= 0 || !(max_diff >= 0.0f)) return OR_ERR_ARG;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const i64 i = (i64)y * W + x;
            const float d = ul[i];
            int pass = 0;
            if (isfinite(d) && fabsf(d) < 1.0e9f) {
                const i64 xr = (i64)x - (i64)rintf(d);
                if (xr >= 0 && xr < W) {
                    const float diff = fabsf(d - ur[(i64)y * W + xr]);
                    pass = diff <= max_diff;
                }
            }
            ok[i] = (uint8_t)pass;
            out[i] = pass ? d : -1.0f;
        }
    return OR_OK;
}

/* Edge strengths omega_ij (Sec. 2.1: image dependent, smaller across sharp
 * edges; reading R3).  wh[y][x] is the edge (y,x)-(y,x+1), wv[y][x] the edge
 * (y,x)-(y+1,x); entries without an edge are 0. */
int or_edge_weights(int H, int W, const uint8_t* img, int T, int w_hi, int w_lo,
                    int32_t* wh, int32_t* wv)
{
    if (H <= 0 || W <= 0) return OR_ERR_ARG;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int i = y * W + x;
            wh[i] = 0;
            wv[i] = 0;
            if (x + 1 < W) wh[i] = abs((int)img[i] - (int)img[i + 1]) < T ? w_hi : w_lo;
            if (y + 1 < H) wv[i] = abs((int)img[i] - (int)img[i + W]) < T ? w_hi : w_lo;
        }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Penalty r (Eq. r-decompose): r = r_{eps,delta} - r_{0, C + delta - eps     */
/* delta}, r_{a,b}(t) = a|t| if |t| <= b else |t| - b(1-a).                   */
/* ------------------------------------------------------------------------ */

double or_r_ab(double t, double a, double b)
{
    double at = fabs(t);
    return at <= b ? a * at : at - b * (1.0 - a);
}

double or_r(double t, double eps, double delta, double C)
{
    return or_r_ab(t, eps, delta) - or_r_ab(t, 0.0, C + delta - eps * delta);
}

/* V[t] = omega * r(t), t = 0..K-1, sampled at integer label distances
 * (Sec. 2.2: f_ij = omega_ij r((Au(x))_ij); Fig. 2).  Fails if not integer. */
int or_penalty_table(int omega, double eps, double delta, double C, int K, i64* V)
{
    for (int t = 0; t < K; ++t) {
        double v = (double)omega * or_r((double)t, eps, delta, C);
        double rv = nearbyint(v);
        if (fabs(v - rv) > 1e-9) return OR_ERR_NONINTEGER;
        V[t] = (i64)rv;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Message passing (App. A, Eq. msg-pass; procedure Msg of Alg. Handshake):  */
/*   out(x') = min_x [ a(x) + f_ij(x, x') ],  f_ij(x, x') = V[|x - x'|].      */
/* ------------------------------------------------------------------------ */

void or_msg(int K, const i64* a, const i64* V, i64* out)
{
    for (int xp = 0; xp < K; ++xp) {
        i64 best = INT64_MAX;
        for (int x = 0; x < K; ++x) {
            i64 v = a[x] + V[x > xp ? x - xp : xp - x];
            if (v < best) best = v;
        }
        out[xp] = best;
    }
}

/* Min-marginals of a chain (App. A, Eq. min-marg-expression): left messages
 * phi_{i-1,i}, right messages phi_{i+1,i}, m_i = f_i + phi_{i-1,i} + phi_{i+1,i}.
 * theta: n*K unaries; V: (n-1)*K tables, row k for the edge (k, k+1). */
void or_min_marginals(int n, int K, const i64* theta, const i64* V, i64* mm)
{
    i64* left = (i64*)calloc((size_t)n * K, sizeof(i64));
    i64* right = (i64*)calloc((size_t)n * K, sizeof(i64));
    i64* tmp = (i64*)malloc((size_t)K * sizeof(i64));
    for (int k = 1; k < n; ++k) {
        for (int l = 0; l < K; ++l) tmp[l] = left[(i64)(k - 1) * K + l] + theta[(i64)(k - 1) * K + l];
        or_msg(K, tmp, V + (i64)(k - 1) * K, left + (i64)k * K);
    }
    for (int k = n - 2; k >= 0; --k) {
        for (int l = 0; l < K; ++l) tmp[l] = right[(i64)(k + 1) * K + l] + theta[(i64)(k + 1) * K + l];
        or_msg(K, tmp, V + (i64)k * K, right + (i64)k * K);
    }
    for (i64 e = 0; e < (i64)n * K; ++e) mm[e] = theta[e] + left[e] + right[e];
    free(left);
    free(right);
    free(tmp);
}

/* ------------------------------------------------------------------------ */
/* Hierarchical minorant (App. A "Hierarchical Minorants", Alg. Handshake).  */
/* rec(a, b, Lin, Rin): the sub-chain a..b with the message Lin entering a    */
/* from the left and Rin entering b from the right.                           */
/* ------------------------------------------------------------------------ */

static i64 floor_half(i64 m) { return m >= 0 ? m / 2 : -((-m + 1) / 2); }

static void hier_rec(int a, int b, int K, const i64* theta, const i64* V, const i64* Lin,
                     const i64* Rin, i64* lam)
{
    if (a == b) {
        /* a single node keeps its whole min-marginal (reading R6) */
        for (int l = 0; l < K; ++l) lam[(i64)a * K + l] = theta[(i64)a * K + l] + Lin[l] + Rin[l];
        return;
    }
    int len = b - a + 1;
    int i = a + (len + 1) / 2 - 1; /* left part keeps ceil(len/2) nodes */
    int j = i + 1;
    i64* Lm = (i64*)malloc((size_t)K * sizeof(i64));
    i64* Rm = (i64*)malloc((size_t)K * sizeof(i64));
    i64* tmp = (i64*)malloc((size_t)K * sizeof(i64));
    i64* phi_ji = (i64*)malloc((size_t)K * sizeof(i64));
    i64* phi_ij = (i64*)malloc((size_t)K * sizeof(i64));
    i64* m_i = (i64*)malloc((size_t)K * sizeof(i64));

    /* left min-marginal message into i: sweep a .. i-1 */
    memcpy(Lm, Lin, (size_t)K * sizeof(i64));
    for (int k = a; k < i; ++k) {
        for (int l = 0; l < K; ++l) tmp[l] = theta[(i64)k * K + l] + Lm[l];
        or_msg(K, tmp, V + (i64)k * K, Lm);
    }
    /* right min-marginal message into j: sweep b .. j+1 */
    memcpy(Rm, Rin, (size_t)K * sizeof(i64));
    for (int k = b; k > j; --k) {
        for (int l = 0; l < K; ++l) tmp[l] = theta[(i64)k * K + l] + Rm[l];
        or_msg(K, tmp, V + (i64)(k - 1) * K, Rm);
    }
    /* Handshake over the edge (i, j) */
    for (int l = 0; l < K; ++l) tmp[l] = theta[(i64)j * K + l] + Rm[l];
    or_msg(K, tmp, V + (i64)i * K, phi_ji);                  /* message j -> i        */
    for (int l = 0; l < K; ++l)
        m_i[l] = Lm[l] + theta[(i64)i * K + l] + phi_ji[l];  /* total min-marginal at i */
    for (int l = 0; l < K; ++l) tmp[l] = floor_half(m_i[l]) - phi_ji[l];
    or_msg(K, tmp, V + (i64)i * K, phi_ij);                  /* share a half to the right */
    for (int l = 0; l < K; ++l) tmp[l] = -phi_ij[l];
    or_msg(K, tmp, V + (i64)i * K, phi_ji);                  /* bounce back the rest   */

    hier_rec(a, i, K, theta, V, Lin, phi_ji, lam);
    hier_rec(j, b, K, theta, V, phi_ij, Rin, lam);
    free(Lm); free(Rm); free(tmp); free(phi_ji); free(phi_ij); free(m_i);
}

/* lam = hierarchical minorant of the chain (theta, V) with zero boundary messages */
void or_hier_minorant(int n, int K, const i64* theta, const i64* V, i64* lam)
{
    i64* zero = (i64*)calloc((size_t)K, sizeof(i64));
    hier_rec(0, n - 1, K, theta, V, zero, zero, lam);
    free(zero);
}

/* ------------------------------------------------------------------------ */
/* Other minorants of a chain (Sec. 2.3 "Good and Fast Minorants"; App. A).  */
/* ------------------------------------------------------------------------ */

/* floor(a / d) for d > 0 */
static i64 floor_div(i64 a, i64 d) { return a >= 0 ? a / d : -((-a + d - 1) / d); }

/* Naive minorant: every node takes its min-marginal of the chain divided by
 * the chain length n (reading R29: rounded down, so that the sum over the
 * nodes stays below f). */
void or_naive_minorant(int n, int K, const i64* theta, const i64* V, i64* lam)
{
    or_min_marginals(n, K, theta, V, lam);
    for (i64 e = 0; e < (i64)n * K; ++e) lam[e] = floor_div(lam[e], n);
}

/* Iterative minorant (Alg. iterative-minorant; reading R30).  lam starts at 0.
 * Pass s = 1..max_pass visits the nodes forward (s odd) or backward (s even);
 * at node i the min-marginal of the remainder f - lam is the message entering
 * i from the side visited earlier in this pass (Eq. msg-pass, formed with the
 * nodes already updated), plus theta_i - lam_i, plus the message entering from
 * the other side, left by the previous pass (an initial backward sweep before
 * the first pass); then lam_i += floor(gamma_s m_i), gamma_s = gn/gd for
 * s < max_pass and 1 for the last pass. */
int or_iterative_minorant(int n, int K, const i64* theta, const i64* V, int max_pass, int gn,
                          int gd, i64* lam)
{
    if (n <= 0 || K <= 0 || max_pass < 1 || gn < 0 || gd <= 0 || gn > gd) return OR_ERR_ARG;
    i64* left = (i64*)calloc((size_t)n * K, sizeof(i64));   /* left[i]: message (i-1 -> i)  */
    i64* right = (i64*)calloc((size_t)n * K, sizeof(i64));  /* right[i]: message (i+1 -> i) */
    i64* tmp = (i64*)malloc((size_t)K * sizeof(i64));
    memset(lam, 0, (size_t)n * K * sizeof(i64));
    for (int k = n - 2; k >= 0; --k) {
        for (int l = 0; l < K; ++l)
            tmp[l] = theta[(i64)(k + 1) * K + l] - lam[(i64)(k + 1) * K + l] + right[(i64)(k + 1) * K + l];
        or_msg(K, tmp, V + (i64)k * K, right + (i64)k * K);
    }
    for (int s = 1; s <= max_pass; ++s) {
        const i64 num = s == max_pass ? 1 : gn, den = s == max_pass ? 1 : gd;
        const int fwd = (s & 1) == 1;
        for (int t = 0; t < n; ++t) {
            const int i = fwd ? t : n - 1 - t;
            if (fwd) {
                if (i == 0) memset(left, 0, (size_t)K * sizeof(i64));
                else {
                    for (int l = 0; l < K; ++l)
                        tmp[l] = theta[(i64)(i - 1) * K + l] - lam[(i64)(i - 1) * K + l] +
                                 left[(i64)(i - 1) * K + l];
                    or_msg(K, tmp, V + (i64)(i - 1) * K, left + (i64)i * K);
                }
            } else {
                if (i == n - 1) memset(right + (i64)(n - 1) * K, 0, (size_t)K * sizeof(i64));
                else {
                    for (int l = 0; l < K; ++l)
                        tmp[l] = theta[(i64)(i + 1) * K + l] - lam[(i64)(i + 1) * K + l] +
                                 right[(i64)(i + 1) * K + l];
                    or_msg(K, tmp, V + (i64)i * K, right + (i64)i * K);
                }
            }
            for (int l = 0; l < K; ++l) {
                const i64 e = (i64)i * K + l;
                const i64 m = left[e] + theta[e] - lam[e] + right[e];
                lam[e] += floor_div(m * num, den);
            }
        }
    }
    free(left); free(right); free(tmp);
    return OR_OK;
}

/* Minimum of the chain (theta, V) and a minimiser (plain forward recursion with
 * back-pointers, Eq. msg-pass); x may be NULL. */
static double chain_viterbi(int n, int K, const double* theta, const i64* V, int* x)
{
    double* best = (double*)malloc((size_t)n * K * sizeof(double));
    int* arg = (int*)malloc((size_t)n * K * sizeof(int));
    for (int l = 0; l < K; ++l) best[l] = theta[l];
    for (int k = 1; k < n; ++k)
        for (int b = 0; b < K; ++b) {
            double m = INFINITY;
            int am = 0;
            for (int a = 0; a < K; ++a) {
                double v = best[(i64)(k - 1) * K + a] + (double)V[(i64)(k - 1) * K + (a > b ? a - b : b - a)];
                if (v < m) { m = v; am = a; }
            }
            best[(i64)k * K + b] = m + theta[(i64)k * K + b];
            arg[(i64)k * K + b] = am;
        }
    double m = INFINITY;
    int l_end = 0;
    for (int l = 0; l < K; ++l)
        if (best[(i64)(n - 1) * K + l] < m) { m = best[(i64)(n - 1) * K + l]; l_end = l; }
    if (x) {
        x[n - 1] = l_end;
        for (int k = n - 1; k > 0; --k) x[k - 1] = arg[(i64)k * K + x[k]];
    }
    free(best);
    free(arg);
    return m;
}

/* Maximal uniform minorant (Alg. uniform-minorant; reading R38).  lam := 0;
 * repeat: min-marginals m of f - lam; stop when all vanish (|m| <= tol);
 * O = [m <= tol]; eps = min over labellings x with <1-O, x> > 0 of
 * (f - lam)(x) / <1-O, x>, the minimum ratio path of Lawler's method, found by
 * Dinkelbach's parametric iteration (a Viterbi pass of f - lam - eps (1-O) per
 * step); lam += eps (1-O).  Double precision; returns the number of rounds
 * (or -1 without convergence within max_rounds). */
int or_uniform_minorant(int n, int K, const i64* theta, const i64* V, double tol, int max_rounds,
                        double* lam)
{
    double* rem = (double*)malloc((size_t)n * K * sizeof(double));   /* theta - lam */
    double* t2 = (double*)malloc((size_t)n * K * sizeof(double));
    double* left = (double*)malloc((size_t)n * K * sizeof(double));
    double* right = (double*)malloc((size_t)n * K * sizeof(double));
    double* mm = (double*)malloc((size_t)n * K * sizeof(double));
    int* O = (int*)malloc((size_t)n * K * sizeof(int));
    int* x = (int*)malloc((size_t)n * sizeof(int));
    int rounds = -1;
    for (i64 e = 0; e < (i64)n * K; ++e) lam[e] = 0.0;
    for (int r = 0; r < max_rounds; ++r) {
        for (i64 e = 0; e < (i64)n * K; ++e) rem[e] = (double)theta[e] - lam[e];
        /* min-marginals of the remainder (Eq. min-marg-expression) */
        for (int l = 0; l < K; ++l) { left[l] = 0.0; right[(i64)(n - 1) * K + l] = 0.0; }
        for (int k = 1; k < n; ++k)
            for (int b = 0; b < K; ++b) {
                double m = INFINITY;
                for (int a = 0; a < K; ++a) {
                    double v = left[(i64)(k - 1) * K + a] + rem[(i64)(k - 1) * K + a] +
                               (double)V[(i64)(k - 1) * K + (a > b ? a - b : b - a)];
                    if (v < m) m = v;
                }
                left[(i64)k * K + b] = m;
            }
        for (int k = n - 2; k >= 0; --k)
            for (int a = 0; a < K; ++a) {
                double m = INFINITY;
                for (int b = 0; b < K; ++b) {
                    double v = right[(i64)(k + 1) * K + b] + rem[(i64)(k + 1) * K + b] +
                               (double)V[(i64)k * K + (a > b ? a - b : b - a)];
                    if (v < m) m = v;
                }
                right[(i64)k * K + a] = m;
            }
        int all_zero = 1;
        for (i64 e = 0; e < (i64)n * K; ++e) {
            mm[e] = left[e] + rem[e] + right[e];
            O[e] = fabs(mm[e]) <= tol;
            if (!O[e]) all_zero = 0;
        }
        if (all_zero) { rounds = r; break; }
        /* Dinkelbach: start from the ratio of a minimiser of f - lam that uses a
         * label outside O (one exists: some min-marginal is positive) */
        double eps = INFINITY;
        {
            /* the labelling that takes, at the first node with a non-optimal label,
             * that label and the best completion: its ratio is finite */
            for (i64 e = 0; e < (i64)n * K; ++e) t2[e] = rem[e] - (O[e] ? 0.0 : 1e6);
            chain_viterbi(n, K, t2, V, x);
            double A = 0.0, Bc = 0.0;
            for (int k = 0; k < n; ++k) {
                A += rem[(i64)k * K + x[k]];
                Bc += O[(i64)k * K + x[k]] ? 0.0 : 1.0;
                if (k + 1 < n) A += (double)V[(i64)k * K + (x[k] > x[k + 1] ? x[k] - x[k + 1] : x[k + 1] - x[k])];
            }
            eps = A / Bc;
        }
        for (int it = 0; it < 200; ++it) {
            for (i64 e = 0; e < (i64)n * K; ++e) t2[e] = rem[e] - (O[e] ? 0.0 : eps);
            double v = chain_viterbi(n, K, t2, V, x);
            if (v >= -tol) break;   /* min_x A - eps B = 0: eps is the minimum ratio */
            double A = 0.0, Bc = 0.0;
            for (int k = 0; k < n; ++k) {
                A += rem[(i64)k * K + x[k]];
                Bc += O[(i64)k * K + x[k]] ? 0.0 : 1.0;
                if (k + 1 < n) A += (double)V[(i64)k * K + (x[k] > x[k + 1] ? x[k] - x[k + 1] : x[k + 1] - x[k])];
            }
            eps = A / Bc;
        }
        for (i64 e = 0; e < (i64)n * K; ++e)
            if (!O[e]) lam[e] += eps;
    }
    free(rem); free(t2); free(left); free(right); free(mm); free(O); free(x);
    return rounds;
}

/* ------------------------------------------------------------------------ */
/* Dual MM (Alg. Dual_MM) on the 4-connected grid split into horizontal      */
/* chains f (data cost + horizontal edges) and vertical chains g (vertical    */
/* edges only).  lam_h is the minorant f^{k+1} of f, lam_v the minorant g^k.  */
/* ------------------------------------------------------------------------ */

typedef struct {
    i64* table[256];   /* omega -> K entries (built on first use) */
} or_tables;

static int build_tables(or_tables* T, int K, const int32_t* w, int count, double eps,
                        double delta, double C)
{
    for (int t = 0; t < 256; ++t) T->table[t] = NULL;
    for (int e = 0; e < count; ++e) {
        int om = w[e];
        if (om < 0 || om > 255) return OR_ERR_ARG;
        if (T->table[om]) continue;
        T->table[om] = (i64*)malloc((size_t)K * sizeof(i64));
        int rc = or_penalty_table(om, eps, delta, C, K, T->table[om]);
        if (rc) return rc;
    }
    return OR_OK;
}

static const i64* find_table(const or_tables* T, int om) { return T->table[om]; }

static void free_tables(or_tables* T)
{
    for (int t = 0; t < 256; ++t) free(T->table[t]);
}

/* One pass of Alg. Dual_MM.
 *   which = 0 (horizontal): theta = cost + lam_in (lam_in = lam_v),
 *             mu = minorant(theta), lam_out = mu - lam_in   (steps 1-2)
 *   which = 1 (vertical):   theta = lam_in (lam_in = lam_h),
 *             nu = minorant(theta), lam_out = nu - lam_in   (steps 3-4)
 * kind: 0 hierarchical (App. A), 1 naive, 2 iterative (max_pass, gn/gd). */
int or_dmm_pass_kind(int H, int W, int L, const int32_t* cost, const int32_t* wh,
                     const int32_t* wv, double eps, double delta, double C, int which,
                     const i64* lam_in, i64* lam_out, int nthreads, int kind, int max_pass,
                     int gn, int gd)
{
    if (H <= 0 || W <= 0 || L <= 0 || (which != 0 && which != 1)) return OR_ERR_ARG;
    if (kind < 0 || kind > 2) return OR_ERR_ARG;
    if (kind == 2 && (max_pass < 1 || gn < 0 || gd <= 0 || gn > gd)) return OR_ERR_ARG;
    or_tables T;
    int rc = build_tables(&T, L, which == 0 ? wh : wv, H * W, eps, delta, C);
    if (rc) { free_tables(&T); return rc; }
    int nchains = which == 0 ? H : W;
    int n = which == 0 ? W : H;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int c = 0; c < nchains; ++c) {
        i64* theta = (i64*)malloc((size_t)n * L * sizeof(i64));
        i64* V = (i64*)malloc((size_t)(n > 1 ? n - 1 : 1) * L * sizeof(i64));
        i64* mu = (i64*)malloc((size_t)n * L * sizeof(i64));
        for (int k = 0; k < n; ++k) {
            int y = which == 0 ? c : k, x = which == 0 ? k : c;
            i64 pix = (i64)y * W + x;
            for (int l = 0; l < L; ++l) {
                i64 t = lam_in[pix * L + l];
                if (which == 0) t += cost[pix * L + l];
                theta[(i64)k * L + l] = t;
            }
            if (k + 1 < n) {
                const i64* tab = find_table(&T, which == 0 ? wh[pix] : wv[pix]);
                memcpy(V + (i64)k * L, tab, (size_t)L * sizeof(i64));
            }
        }
        if (kind == 0) or_hier_minorant(n, L, theta, V, mu);
        else if (kind == 1) or_naive_minorant(n, L, theta, V, mu);
        else or_iterative_minorant(n, L, theta, V, max_pass, gn, gd, mu);
        for (int k = 0; k < n; ++k) {
            int y = which == 0 ? c : k, x = which == 0 ? k : c;
            i64 pix = (i64)y * W + x;
            for (int l = 0; l < L; ++l)
                lam_out[pix * L + l] = mu[(i64)k * L + l] - lam_in[pix * L + l];
        }
        free(theta); free(V); free(mu);
    }
    free_tables(&T);
    return OR_OK;
}

int or_dmm_pass(int H, int W, int L, const int32_t* cost, const int32_t* wh,
                const int32_t* wv, double eps, double delta, double C, int which,
                const i64* lam_in, i64* lam_out, int nthreads)
{
    return or_dmm_pass_kind(H, W, L, cost, wh, wv, eps, delta, C, which, lam_in, lam_out,
                            nthreads, 0, 1, 1, 1);
}

/* Labels and lower bound from the two minorants (weak duality, Eq. DD-dual;
 * readings R7). */
i64 or_dmm_outputs(int H, int W, int L, const i64* lam_h, const i64* lam_v, uint16_t* labels)
{
    i64 lb = 0;
    for (i64 p = 0; p < (i64)H * W; ++p) {
        i64 best = INT64_MAX;
        int arg = 0;
        for (int l = 0; l < L; ++l) {
            i64 v = lam_h[p * L + l] + lam_v[p * L + l];
            if (v < best) { best = v; arg = l; }
        }
        lb += best;
        if (labels) labels[p] = (uint16_t)arg;
    }
    return lb;
}

/* Full Dual MM: iters x (horizontal pass, vertical pass), starting from the
 * given lam_v (zero for a cold start).  lb[t] is the bound after iteration t. */
int or_dmm_kind(int H, int W, int L, const int32_t* cost, const int32_t* wh,
                const int32_t* wv, double eps, double delta, double C, int iters, i64* lam_h,
                i64* lam_v, i64* lb, uint16_t* labels, int nthreads, int kind, int max_pass,
                int gn, int gd)
{
    for (int t = 0; t < iters; ++t) {
        int rc = or_dmm_pass_kind(H, W, L, cost, wh, wv, eps, delta, C, 0, lam_v, lam_h,
                                  nthreads, kind, max_pass, gn, gd);
        if (rc) return rc;
        rc = or_dmm_pass_kind(H, W, L, cost, wh, wv, eps, delta, C, 1, lam_h, lam_v, nthreads,
                              kind, max_pass, gn, gd);
        if (rc) return rc;
        i64 b = or_dmm_outputs(H, W, L, lam_h, lam_v, (t == iters - 1) ? labels : NULL);
        if (lb) lb[t] = b;
    }
    return OR_OK;
}

int or_dmm(int H, int W, int L, const int32_t* cost, const int32_t* wh, const int32_t* wv,
           double eps, double delta, double C, int iters, i64* lam_h, i64* lam_v, i64* lb,
           uint16_t* labels, int nthreads)
{
    return or_dmm_kind(H, W, L, cost, wh, wv, eps, delta, C, iters, lam_h, lam_v, lb, labels,
                       nthreads, 0, 1, 1, 1);
}

/* The modular majorant of Primal_MM exact at `labels` (reading R39): half 0
 * majorises f (the data cost and the horizontal edges), half 1 majorises g
 * (the vertical edges).  bar[p][l] = (data cost if half 0) + sum over the
 * family's edges at p of f_e(labels)/2 + cap_e [l != labels_p], cap_e =
 * max_d omega_e r(d); then sum_p bar[p][x_p] >= the family's energy at x with
 * equality at x = labels. */
static void pmm_majorant(int H, int W, int L, const int32_t* cost, const int32_t* wh,
                         const int32_t* wv, const or_tables* T, int half, const uint16_t* labels,
                         double* bar)
{
    for (int y = 0; y < H; ++y)
        for (int xx = 0; xx < W; ++xx) {
            i64 p = (i64)y * W + xx;
            for (int l = 0; l < L; ++l) bar[p * L + l] = half == 0 ? (double)cost[p * L + l] : 0.0;
        }
    for (int y = 0; y < H; ++y)
        for (int xx = 0; xx < W; ++xx) {
            i64 p = (i64)y * W + xx;
            int has = half == 0 ? xx + 1 < W : y + 1 < H;
            if (!has) continue;
            i64 q = half == 0 ? p + 1 : p + W;
            int om = half == 0 ? wh[p] : wv[p];
            const i64* tab = find_table(T, om);
            double cap = 0.0;
            for (int d = 0; d < L; ++d) if ((double)tab[d] > cap) cap = (double)tab[d];
            int a = labels[p], b = labels[q];
            double cur = (double)tab[a > b ? a - b : b - a];
            for (int l = 0; l < L; ++l) {
                bar[p * L + l] += 0.5 * cur + (l != a ? cap : 0.0);
                bar[q * L + l] += 0.5 * cur + (l != b ? cap : 0.0);
            }
        }
}

/* The majorant alone (for its pin): bar [H][W][L] of the family `half` at labels. */
int or_pmm_majorant(int H, int W, int L, const int32_t* cost, const int32_t* wh, const int32_t* wv,
                    double eps, double delta, double C, int half, const uint16_t* labels, double* bar)
{
    if (H <= 0 || W <= 0 || L <= 0 || (half != 0 && half != 1)) return OR_ERR_ARG;
    or_tables T;
    int rc = build_tables(&T, L, half == 0 ? wh : wv, H * W, eps, delta, C);
    if (!rc) pmm_majorant(H, W, L, cost, wh, wv, &T, half, labels, bar);
    free_tables(&T);
    return rc;
}

/* Primal_MM (Alg. Primal_MM) on the grid split into horizontal chains f (data
 * and horizontal edges) and vertical chains g.  The modular majorant of a chain
 * exact at the current labelling xk (reading R39): every edge (i, j) charges
 * omega C (the cap of its truncated penalty) to each end whose label leaves xk,
 * and splits its current cost f_ij(xk_i, xk_j) evenly between the two ends;
 * since 0 <= f_ij <= omega C this is >= f_ij everywhere and equal at xk.
 * One iteration: majorise f at xk, minimise the vertical chains g + f_bar;
 * majorise g at the result, minimise the horizontal chains f + g_bar.
 * labels: the start on entry, the result on exit; energy[t] after iteration t. */
i64 or_discrete_energy(int H, int W, int L, const int32_t* cost, const int32_t* wh,
                       const int32_t* wv, double eps, double delta, double C,
                       const uint16_t* labels);

int or_primal_mm(int H, int W, int L, const int32_t* cost, const int32_t* wh, const int32_t* wv,
                 double eps, double delta, double C, int iters, uint16_t* labels, i64* energy)
{
    if (H <= 0 || W <= 0 || L <= 0 || iters < 0) return OR_ERR_ARG;
    or_tables Th, Tv;
    int rc = build_tables(&Th, L, wh, H * W, eps, delta, C);
    if (!rc) rc = build_tables(&Tv, L, wv, H * W, eps, delta, C);
    if (rc) { free_tables(&Th); return rc; }
    const int n = H > W ? H : W;
    double* theta = (double*)malloc((size_t)n * L * sizeof(double));
    i64* V = (i64*)malloc((size_t)n * L * sizeof(i64));
    int* x = (int*)malloc((size_t)n * sizeof(int));
    double* bar = (double*)malloc((size_t)H * W * L * sizeof(double));
    for (int t = 0; t < iters; ++t) {
        for (int half = 0; half < 2; ++half) {
            /* half 0: majorise f (horizontal edges + data), minimise columns of g + f_bar;
             * half 1: majorise g (vertical edges), minimise rows of f + g_bar */
            pmm_majorant(H, W, L, cost, wh, wv, half == 0 ? &Th : &Tv, half, labels, bar);
            /* minimise the other family of chains plus the modular majorant */
            int nch = half == 0 ? W : H, len = half == 0 ? H : W;
            for (int c = 0; c < nch; ++c) {
                for (int k = 0; k < len; ++k) {
                    int y = half == 0 ? k : c, xx = half == 0 ? c : k;
                    i64 p = (i64)y * W + xx;
                    for (int l = 0; l < L; ++l) {
                        double v = bar[p * L + l];
                        if (half == 1) v += (double)cost[p * L + l];
                        theta[(i64)k * L + l] = v;
                    }
                    if (k + 1 < len) {
                        int om = half == 0 ? wv[p] : wh[p];
                        memcpy(V + (i64)k * L, find_table(half == 0 ? &Tv : &Th, om),
                               (size_t)L * sizeof(i64));
                    }
                }
                chain_viterbi(len, L, theta, V, x);
                for (int k = 0; k < len; ++k) {
                    int y = half == 0 ? k : c, xx = half == 0 ? c : k;
                    labels[(i64)y * W + xx] = (uint16_t)x[k];
                }
            }
        }
        if (energy) energy[t] = or_discrete_energy(H, W, L, cost, wh, wv, eps, delta, C, labels);
    }
    free(theta); free(V); free(x); free(bar);
    free_tables(&Th); free_tables(&Tv);
    return OR_OK;
}

/* Discrete energy, Eq. (energy-pairwise) with the stereo terms of Sec. 2.2. */
i64 or_discrete_energy(int H, int W, int L, const int32_t* cost, const int32_t* wh,
                       const int32_t* wv, double eps, double delta, double C,
                       const uint16_t* labels)
{
    i64 e = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            i64 p = (i64)y * W + x;
            int xi = labels[p];
            e += cost[p * L + xi];
            if (x + 1 < W)
                e += (i64)nearbyint(wh[p] * or_r((double)(xi - labels[p + 1]), eps, delta, C));
            if (y + 1 < H)
                e += (i64)nearbyint(wv[p] * or_r((double)(xi - labels[p + W]), eps, delta, C));
        }
    return e;
}

/* ------------------------------------------------------------------------ */
/* Continuous refinement (Sec. 2.4 and 3.1), double precision.               */
/* ------------------------------------------------------------------------ */

/* D_i(u): piecewise-linear interpolation of the samples c[0..L-1] (reading R8) */
double or_interp(int L, const double* c, double u)
{
    if (u <= 0.0) return c[0];
    if (u >= (double)(L - 1)) return c[L - 1];
    double fl = floor(u);
    int k = (int)fl;
    double t = u - fl;
    return c[k] + t * (c[k + 1] - c[k]);
}

/* Linearisation of the data term around u0 (Sec. 3.1; readings R9):
 * slopes s1 (left of u0), s2 (right of u0), box [lo, hi]. */
void or_linearise_px(int L, const double* c, double alpha, double u0, double h, double* s1,
                     double* s2, double* lo, double* hi)
{
    double d0 = or_interp(L, c, u0);
    double dm = or_interp(L, c, u0 - h);
    double dp = or_interp(L, c, u0 + h);
    double a = alpha * (d0 - dm) / h;
    double b = alpha * (dp - d0) / h;
    if (b < a) { a = 0.5 * (a + b); b = a; }
    *s1 = a;
    *s2 = b;
    *lo = u0 - h > 0.0 ? u0 - h : 0.0;
    *hi = u0 + h < (double)(L - 1) ? u0 + h : (double)(L - 1);
}

/* prox of tau * D~ at uh (Sec. 3.1, pointwise soft-threshold; reading R10) */
double or_prox_data(double uh, double u0, double s1, double s2, double lo, double hi,
                    double tau)
{
    double v;
    if (uh > u0 + tau * s2) v = uh - tau * s2;
    else if (uh < u0 + tau * s1) v = uh - tau * s1;
    else v = u0;
    if (v < lo) v = lo;
    if (v > hi) v = hi;
    return v;
}

/* prox of step * (omega r_{a,b})* at t (Eq. pprox; reading R11):
 * t' = t if |t| <= a*omega, else sign(t) max(a*omega, |t| - b*step); clamp to +-omega */
double or_prox_conj(double t, double omega, double a, double b, double step)
{
    double tp;
    if (fabs(t) <= a * omega) tp = t;
    else {
        double m = fabs(t) - b * step;
        if (m < a * omega) m = a * omega;
        tp = t > 0 ? m : -m;
    }
    if (tp > omega) tp = omega;
    if (tp < -omega) tp = -omega;
    return tp;
}

/* convex conjugate (omega r_{a,b})*(s) (reading R11); +inf outside |s| <= omega */
double or_conj(double s, double omega, double a, double b)
{
    if (fabs(s) > omega * (1.0 + 1e-12)) return INFINITY;
    double v = fabs(s) - omega * a;
    return v > 0 ? b * v : 0.0;
}

typedef struct {
    double eps, delta, C;   /* penalty r */
    double lambda_r;        /* regulariser weight (multiplies omega) */
    double tau, sigma, h;   /* primal / dual steps, linearisation half-width */
    int warps;              /* re-linearisations (warping) */
} or_cont_params;

/* Continuous energy E(u) = sum_i alpha_i D_i(u_i) + sum_e lambda_r omega_e r((Au)_e)
 * (Eq. mrf_formulation, regularizer-form). */
double or_cont_energy(int H, int W, int L, const double* cost, const double* alpha,
                      const double* wh, const double* wv, const or_cont_params* P,
                      const double* u)
{
    double e = 0.0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            i64 p = (i64)y * W + x;
            double a = alpha ? alpha[p] : 1.0;
            e += a * or_interp(L, cost + p * L, u[p]);
            if (x + 1 < W) e += P->lambda_r * wh[p] * or_r(u[p] - u[p + 1], P->eps, P->delta, P->C);
            if (y + 1 < H) e += P->lambda_r * wv[p] * or_r(u[p] - u[p + W], P->eps, P->delta, P->C);
        }
    return e;
}

/* Non-linear primal-dual refinement (Eq. cont_iterates with the operator of
 * Eq. cont_problem, nabla A of Sec. 2.4, data term of Sec. 3.1).
 *   A u on the edge e = (i, j) (i left/top, j right/bottom) is u_i - u_j.
 *   u  <- prox_{tau D~}(u - tau A^T (p - q))
 *   q  <- prox_{tau R-*}(q + tau A u_old)
 *   p  <- prox_{sigma R+*}(p + sigma A (2 u_new - u_old))
 * with R+ = sum lambda_r omega r_{eps,delta}, R- = sum lambda_r omega r_{0,C+delta-eps delta}.
 * State arrays are H*W (edge arrays store the edge at its left/top pixel; the
 * last column of *_h and last row of *_v are unused and kept at 0).
 * If init is nonzero, p and q are reset to 0 first; u holds u0 on entry.
 * energy (nullable): E(u) after each warp.
 * noise > 0 (or_refine_perturbed only): after every iteration each of u, p and
 * q is multiplied by 1 + noise * U, U uniform in [-1, 1) from splitmix64. */
static int refine_run(int H, int W, int L, const double* cost, const double* alpha, const double* wh,
                      const double* wv, int iters, const or_cont_params* P, double* u, double* ph,
                      double* pv, double* qh, double* qv, int init, double* energy, double noise,
                      uint64_t seed);

int or_refine(int H, int W, int L, const double* cost, const double* alpha, const double* wh,
              const double* wv, int iters, const or_cont_params* P, double* u, double* ph,
              double* pv, double* qh, double* qv, int init, double* energy)
{
    return refine_run(H, W, L, cost, alpha, wh, wv, iters, P, u, ph, pv, qh, qv, init, energy,
                      0.0, 0);
}

/* splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the finaliser applied to seed + (n + 1) * golden
 * gamma, i.e. the n-th output of the generator started at seed; mapped to
 * [-1, 1) with 53 bits. */
static double splitmix_unit(uint64_t seed, uint64_t n)
{
    uint64_t z = seed + (n + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

/* The refinement with relative noise of size `noise` put on the state (u, p,
 * q) after every iteration: a model of rounding the state to a shorter float
 * (2^-24 for float32), used to measure how far the double-precision result at
 * each pixel is determined by a computation that carries that precision. */
int or_refine_perturbed(int H, int W, int L, const double* cost, const double* alpha,
                        const double* wh, const double* wv, int iters, const or_cont_params* P,
                        double* u, double* ph, double* pv, double* qh, double* qv, int init,
                        double noise, uint64_t seed)
{
    if (!(noise >= 0.0)) return OR_ERR_ARG;
    return refine_run(H, W, L, cost, alpha, wh, wv, iters, P, u, ph, pv, qh, qv, init, NULL,
                      noise, seed);
}

static int refine_run(int H, int W, int L, const double* cost, const double* alpha, const double* wh,
                      const double* wv, int iters, const or_cont_params* P, double* u, double* ph,
                      double* pv, double* qh, double* qv, int init, double* energy, double noise,
                      uint64_t seed)
{
    if (H <= 0 || W <= 0 || L < 2 || P->warps <= 0) return OR_ERR_ARG;
    i64 N = (i64)H * W;
    double* s1 = (double*)malloc(N * sizeof(double));
    double* s2 = (double*)malloc(N * sizeof(double));
    double* lo = (double*)malloc(N * sizeof(double));
    double* hi = (double*)malloc(N * sizeof(double));
    double* u0 = (double*)malloc(N * sizeof(double));
    double* un = (double*)malloc(N * sizeof(double));
    if (init) {
        for (i64 p = 0; p < N; ++p) ph[p] = pv[p] = qh[p] = qv[p] = 0.0;
    }
    const double bp = P->delta;                              /* beta of R+ */
    const double ap = P->eps;                                /* alpha of R+ */
    const double bq = P->C + P->delta - P->eps * P->delta;   /* beta of R- (alpha = 0) */
    const double tau = P->tau, sigma = P->sigma;
    uint64_t step = 0;   /* iterations done (the noise counter) */
    int base = iters / P->warps, extra = iters % P->warps;
    for (int w = 0; w < P->warps; ++w) {
        int nit = base + (w < extra ? 1 : 0);
        for (i64 p = 0; p < N; ++p) {
            u0[p] = u[p];
            or_linearise_px(L, cost + p * L, alpha ? alpha[p] : 1.0, u0[p], P->h, &s1[p], &s2[p],
                            &lo[p], &hi[p]);
        }
        for (int it = 0; it < nit; ++it) {
            /* primal step for u (uses old p, q) */
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    i64 p = (i64)y * W + x;
                    double div = 0.0; /* (A^T (p - q))_i */
                    if (x + 1 < W) div += ph[p] - qh[p];
                    if (x > 0) div -= ph[p - 1] - qh[p - 1];
                    if (y + 1 < H) div += pv[p] - qv[p];
                    if (y > 0) div -= pv[p - W] - qv[p - W];
                    un[p] = or_prox_data(u[p] - tau * div, u0[p], s1[p], s2[p], lo[p], hi[p], tau);
                }
            /* primal step for q (uses old u) and dual step for p (extrapolated u) */
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    i64 p = (i64)y * W + x;
                    if (x + 1 < W) {
                        double om = P->lambda_r * wh[p];
                        double au = u[p] - u[p + 1];
                        double ext = (2.0 * un[p] - u[p]) - (2.0 * un[p + 1] - u[p + 1]);
                        qh[p] = or_prox_conj(qh[p] + tau * au, om, 0.0, bq, tau);
                        ph[p] = or_prox_conj(ph[p] + sigma * ext, om, ap, bp, sigma);
                    }
                    if (y + 1 < H) {
                        double om = P->lambda_r * wv[p];
                        double au = u[p] - u[p + W];
                        double ext = (2.0 * un[p] - u[p]) - (2.0 * un[p + W] - u[p + W]);
                        qv[p] = or_prox_conj(qv[p] + tau * au, om, 0.0, bq, tau);
                        pv[p] = or_prox_conj(pv[p] + sigma * ext, om, ap, bp, sigma);
                    }
                }
            memcpy(u, un, N * sizeof(double));
            if (noise > 0.0) {
                double* st[5] = {u, ph, pv, qh, qv};
                for (int a = 0; a < 5; ++a)
                    for (i64 p = 0; p < N; ++p)
                        st[a][p] *= 1.0 + noise * splitmix_unit(seed, ((uint64_t)step * 5 + a) * N + p);
                ++step;
            }
        }
        if (energy) energy[w] = or_cont_energy(H, W, L, cost, alpha, wh, wv, P, u);
    }
    free(s1); free(s2); free(lo); free(hi); free(u0); free(un);
    return OR_OK;
}

/* ======================================================================== */
/* Optical flow (Sec. 2.2 "Flow"; the appendix section on optical flow).    */
/* The displacement of pixel (y, x) is (d1, d2), d1 horizontal, d2 vertical, */
/* with d_k = lo_k + label (labels 0..K_k-1; reading R31).                   */
/* ======================================================================== */

typedef struct {
    int H, W, lo1, K1, lo2, K2, maxc;
    const uint32_t* c1;   /* census of I1 */
    const uint32_t* c2;   /* census of I2 */
} or_flow_geo;

/* discretised data cost D_i(d1, d2) = Hamming(census1(y, x), census2(y + d2, x + d1)),
 * maxc where the displaced pixel leaves the image (reading R31) */
static i64 flow_cost_at(const or_flow_geo* G, int y, int x, int d1, int d2)
{
    int yy = y + d2, xx = x + d1;
    if (yy < 0 || yy >= G->H || xx < 0 || xx >= G->W) return G->maxc;
    return popcount32(G->c1[(i64)y * G->W + x] ^ G->c2[(i64)yy * G->W + xx]);
}

/* Decoupled costs (Eq. flow decoupled costs): p1[y][x][l1] = min_l2 D(l1, l2),
 * p2[y][x][l2] = min_l1 D(l1, l2). */
int or_flow_cost_projected(const or_flow_geo* G, int32_t* p1, int32_t* p2)
{
    if (G->H <= 0 || G->W <= 0 || G->K1 <= 0 || G->K2 <= 0) return OR_ERR_ARG;
    for (int y = 0; y < G->H; ++y)
        for (int x = 0; x < G->W; ++x) {
            i64 px = (i64)y * G->W + x;
            for (int a = 0; a < G->K1; ++a) p1[px * G->K1 + a] = INT32_MAX;
            for (int b = 0; b < G->K2; ++b) p2[px * G->K2 + b] = INT32_MAX;
            for (int a = 0; a < G->K1; ++a)
                for (int b = 0; b < G->K2; ++b) {
                    int32_t v = (int32_t)flow_cost_at(G, y, x, G->lo1 + a, G->lo2 + b);
                    if (v < p1[px * G->K1 + a]) p1[px * G->K1 + a] = v;
                    if (v < p2[px * G->K2 + b]) p2[px * G->K2 + b] = v;
                }
        }
    return OR_OK;
}

/* Continuous data term at label coordinates (v1, v2): bilinear interpolation of
 * the integer costs, each argument clamped to [0, K_k - 1] (reading R33). */
double or_flow_D(const or_flow_geo* G, int y, int x, double v1, double v2)
{
    if (v1 < 0.0) v1 = 0.0;
    if (v1 > G->K1 - 1) v1 = G->K1 - 1;
    if (v2 < 0.0) v2 = 0.0;
    if (v2 > G->K2 - 1) v2 = G->K2 - 1;
    int a = (int)floor(v1), b = (int)floor(v2);
    if (a > G->K1 - 2) a = G->K1 - 2 < 0 ? 0 : G->K1 - 2;
    if (b > G->K2 - 2) b = G->K2 - 2 < 0 ? 0 : G->K2 - 2;
    double t = v1 - a, s = v2 - b;
    int a1 = a + 1 < G->K1 ? a + 1 : a, b1 = b + 1 < G->K2 ? b + 1 : b;
    double d00 = (double)flow_cost_at(G, y, x, G->lo1 + a, G->lo2 + b);
    double d10 = (double)flow_cost_at(G, y, x, G->lo1 + a1, G->lo2 + b);
    double d01 = (double)flow_cost_at(G, y, x, G->lo1 + a, G->lo2 + b1);
    double d11 = (double)flow_cost_at(G, y, x, G->lo1 + a1, G->lo2 + b1);
    return (1 - t) * (1 - s) * d00 + t * (1 - s) * d10 + (1 - t) * s * d01 + t * s * d11;
}

/* Quadratic fit (Eq. quadfit) from the 3x3 samples S[j][i] = D(u0 + (i-1) h e1 +
 * (j-1) h e2): L = central first differences, Q = second differences (the mixed
 * term from the four corners), all with step h (reading R35). */
void or_flow_fit_samples(const double* S, double h, double* L, double* Q)
{
    L[0] = (S[1 * 3 + 2] - S[1 * 3 + 0]) / (2.0 * h);
    L[1] = (S[2 * 3 + 1] - S[0 * 3 + 1]) / (2.0 * h);
    Q[0] = (S[1 * 3 + 2] - 2.0 * S[1 * 3 + 1] + S[1 * 3 + 0]) / (h * h);        /* q11 */
    Q[1] = (S[2 * 3 + 2] - S[0 * 3 + 2] - S[2 * 3 + 0] + S[0 * 3 + 0]) / (4.0 * h * h); /* q12 */
    Q[2] = (S[2 * 3 + 1] - 2.0 * S[1 * 3 + 1] + S[0 * 3 + 1]) / (h * h);        /* q22 */
}

/* Positive-semidefinite part of the symmetric 2x2 [[q11, q12], [q12, q22]]: the
 * eigenvalues below zero are set to zero (Werlberger et al.; reading R35). */
void or_psd2(double* Q)
{
    double a = Q[0], b = Q[1], c = Q[2];
    double m = 0.5 * (a + c), r = sqrt(0.25 * (a - c) * (a - c) + b * b);
    double lp = m + r, lm = m - r;
    if (lm >= 0.0) return;
    if (lp <= 0.0) { Q[0] = Q[1] = Q[2] = 0.0; return; }
    /* keep lp v v^T, v the unit eigenvector of lp */
    double v1, v2;
    if (fabs(b) > 0.0) {
        v1 = b; v2 = lp - a;
        if (fabs(v1) + fabs(v2) == 0.0) { v1 = lp - c; v2 = b; }
    } else if (a >= c) { v1 = 1.0; v2 = 0.0; }
    else { v1 = 0.0; v2 = 1.0; }
    double n = sqrt(v1 * v1 + v2 * v2);
    v1 /= n; v2 /= n;
    Q[0] = lp * v1 * v1;
    Q[1] = lp * v1 * v2;
    Q[2] = lp * v2 * v2;
}

/* L, Q (PSD part) of alpha D at u0 and the box, for one pixel */
void or_flow_linearise_px(const or_flow_geo* G, int y, int x, double alpha, double u01,
                          double u02, double h, double* L, double* Q, double* box)
{
    double S[9];
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i)
            S[j * 3 + i] = alpha * or_flow_D(G, y, x, u01 + (i - 1) * h, u02 + (j - 1) * h);
    or_flow_fit_samples(S, h, L, Q);
    or_psd2(Q);
    box[0] = u01 - h > 0.0 ? u01 - h : 0.0;
    box[1] = u01 + h < G->K1 - 1 ? u01 + h : G->K1 - 1;
    box[2] = u02 - h > 0.0 ? u02 - h : 0.0;
    box[3] = u02 + h < G->K2 - 1 ? u02 + h : G->K2 - 1;
}

/* prox of tau D~ for the quadratic model (Eq. prox_flow re-derived, reading R36):
 * u = (I + tau Q)^{-1} (uh + tau (Q u0 - L)), then each component clamped to its box */
void or_flow_prox(double uh1, double uh2, double u01, double u02, const double* L,
                  const double* Q, const double* box, double tau, double* u1, double* u2)
{
    double r1 = uh1 + tau * (Q[0] * u01 + Q[1] * u02 - L[0]);
    double r2 = uh2 + tau * (Q[1] * u01 + Q[2] * u02 - L[1]);
    double m11 = 1.0 + tau * Q[0], m12 = tau * Q[1], m22 = 1.0 + tau * Q[2];
    double det = m11 * m22 - m12 * m12;
    double v1 = (m22 * r1 - m12 * r2) / det;
    double v2 = (m11 * r2 - m12 * r1) / det;
    if (v1 < box[0]) v1 = box[0];
    if (v1 > box[1]) v1 = box[1];
    if (v2 < box[2]) v2 = box[2];
    if (v2 > box[3]) v2 = box[3];
    *u1 = v1;
    *u2 = v2;
}

/* E(u) = sum_i alpha D_i(u_i) + sum_k sum_e lambda_r omega_e r((A u^k)_e) (reading R34) */
double or_flow_energy(const or_flow_geo* G, double alpha, const double* wh, const double* wv,
                      const or_cont_params* P, const double* u1, const double* u2)
{
    double e = 0.0;
    int H = G->H, W = G->W;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            i64 p = (i64)y * W + x;
            e += alpha * or_flow_D(G, y, x, u1[p], u2[p]);
            for (int k = 0; k < 2; ++k) {
                const double* u = k == 0 ? u1 : u2;
                if (x + 1 < W) e += P->lambda_r * wh[p] * or_r(u[p] - u[p + 1], P->eps, P->delta, P->C);
                if (y + 1 < H) e += P->lambda_r * wv[p] * or_r(u[p] - u[p + W], P->eps, P->delta, P->C);
            }
        }
    return e;
}

/* Primal-dual refinement of the flow (Sec. 2.4 iterates, the appendix's
 * quadratic data model): as or_refine, with two components that share the
 * primal prox and have a regulariser each (reading R34, R37).  u1, u2 hold
 * the start (label coordinates) on entry; D (8 arrays: ph1 pv1 qh1 qv1 ph2 pv2
 * qh2 qv2, H*W each) holds the duals; init resets them to 0. */
int or_flow_refine(const or_flow_geo* G, double alpha, const double* wh, const double* wv,
                   int iters, const or_cont_params* P, double* u1, double* u2, double* D, int init,
                   double* energy)
{
    int H = G->H, W = G->W;
    if (H <= 0 || W <= 0 || G->K1 < 2 || G->K2 < 2 || P->warps <= 0) return OR_ERR_ARG;
    i64 N = (i64)H * W;
    double* Lf = (double*)malloc(2 * N * sizeof(double));
    double* Qf = (double*)malloc(3 * N * sizeof(double));
    double* Bx = (double*)malloc(4 * N * sizeof(double));
    double* U0 = (double*)malloc(2 * N * sizeof(double));
    double* un1 = (double*)malloc(N * sizeof(double));
    double* un2 = (double*)malloc(N * sizeof(double));
    if (init) for (i64 e = 0; e < 8 * N; ++e) D[e] = 0.0;
    double* ph[2] = {D, D + 4 * N};
    double* pv[2] = {D + N, D + 5 * N};
    double* qh[2] = {D + 2 * N, D + 6 * N};
    double* qv[2] = {D + 3 * N, D + 7 * N};
    double* u[2] = {u1, u2};
    double* un[2] = {un1, un2};
    const double bp = P->delta, ap = P->eps, bq = P->C + P->delta - P->eps * P->delta;
    const double tau = P->tau, sigma = P->sigma;
    int base = iters / P->warps, extra = iters % P->warps;
    for (int w = 0; w < P->warps; ++w) {
        int nit = base + (w < extra ? 1 : 0);
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                i64 p = (i64)y * W + x;
                U0[2 * p] = u1[p];
                U0[2 * p + 1] = u2[p];
                or_flow_linearise_px(G, y, x, alpha, u1[p], u2[p], P->h, Lf + 2 * p, Qf + 3 * p,
                                     Bx + 4 * p);
            }
        for (int it = 0; it < nit; ++it) {
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    i64 p = (i64)y * W + x;
                    double uh[2];
                    for (int k = 0; k < 2; ++k) {
                        double div = 0.0;
                        if (x + 1 < W) div += ph[k][p] - qh[k][p];
                        if (x > 0) div -= ph[k][p - 1] - qh[k][p - 1];
                        if (y + 1 < H) div += pv[k][p] - qv[k][p];
                        if (y > 0) div -= pv[k][p - W] - qv[k][p - W];
                        uh[k] = u[k][p] - tau * div;
                    }
                    or_flow_prox(uh[0], uh[1], U0[2 * p], U0[2 * p + 1], Lf + 2 * p, Qf + 3 * p,
                                 Bx + 4 * p, tau, &un1[p], &un2[p]);
                }
            for (int k = 0; k < 2; ++k)
                for (int y = 0; y < H; ++y)
                    for (int x = 0; x < W; ++x) {
                        i64 p = (i64)y * W + x;
                        if (x + 1 < W) {
                            double om = P->lambda_r * wh[p];
                            double au = u[k][p] - u[k][p + 1];
                            double ext = (2.0 * un[k][p] - u[k][p]) - (2.0 * un[k][p + 1] - u[k][p + 1]);
                            qh[k][p] = or_prox_conj(qh[k][p] + tau * au, om, 0.0, bq, tau);
                            ph[k][p] = or_prox_conj(ph[k][p] + sigma * ext, om, ap, bp, sigma);
                        }
                        if (y + 1 < H) {
                            double om = P->lambda_r * wv[p];
                            double au = u[k][p] - u[k][p + W];
                            double ext = (2.0 * un[k][p] - u[k][p]) - (2.0 * un[k][p + W] - u[k][p + W]);
                            qv[k][p] = or_prox_conj(qv[k][p] + tau * au, om, 0.0, bq, tau);
                            pv[k][p] = or_prox_conj(pv[k][p] + sigma * ext, om, ap, bp, sigma);
                        }
                    }
            memcpy(u1, un1, N * sizeof(double));
            memcpy(u2, un2, N * sizeof(double));
        }
        if (energy) energy[w] = or_flow_energy(G, alpha, wh, wv, P, u1, u2);
    }
    free(Lf); free(Qf); free(Bx); free(U0); free(un1); free(un2);
    return OR_OK;
}

/* Primal and dual objective of the convex problem obtained when R- vanishes
 * (C -> infinity) for a fixed linearisation (used to check that the
 * primal-dual gap closes).  primal = sum D~_i(u_i) + sum lambda_r omega r_{eps,delta}(Au);
 * dual = -sum D~_i*(-(A^T p)_i) - sum (lambda_r omega r_{eps,delta})*(p).
 * D~_i* is the max over the vertices {lo, u0, hi} of s v - D~_i(v). */
void or_convex_gap(int H, int W, int L, const double* cost, const double* alpha,
                   const double* wh, const double* wv, const or_cont_params* P,
                   const double* u0in, const double* u, const double* ph, const double* pv,
                   double* primal, double* dual)
{
    double pr = 0.0, du = 0.0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            i64 p = (i64)y * W + x;
            double s1, s2, lo, hi;
            double a = alpha ? alpha[p] : 1.0;
            or_linearise_px(L, cost + p * L, a, u0in[p], P->h, &s1, &s2, &lo, &hi);
            double d0 = a * or_interp(L, cost + p * L, u0in[p]);
            /* D~(v) = d0 + s1 (v - u0) for v <= u0, s2 (v - u0) above, +inf outside [lo, hi] */
            double v = u[p];
            double dt = v <= u0in[p] ? d0 + s1 * (v - u0in[p]) : d0 + s2 * (v - u0in[p]);
            if (v < lo - 1e-12 || v > hi + 1e-12) dt = INFINITY;
            pr += dt;
            double atp = 0.0;
            if (x + 1 < W) atp += ph[p];
            if (x > 0) atp -= ph[p - 1];
            if (y + 1 < H) atp += pv[p];
            if (y > 0) atp -= pv[p - W];
            double s = -atp;
            double verts[3] = {lo, u0in[p], hi};
            double best = -INFINITY;
            for (int k = 0; k < 3; ++k) {
                double vv = verts[k];
                double dv = vv <= u0in[p] ? d0 + s1 * (vv - u0in[p]) : d0 + s2 * (vv - u0in[p]);
                double val = s * vv - dv;
                if (val > best) best = val;
            }
            du -= best;
            if (x + 1 < W) {
                double om = P->lambda_r * wh[p];
                pr += om * or_r_ab(u[p] - u[p + 1], P->eps, P->delta);
                du -= or_conj(ph[p], om, P->eps, P->delta);
            }
            if (y + 1 < H) {
                double om = P->lambda_r * wv[p];
                pr += om * or_r_ab(u[p] - u[p + W], P->eps, P->delta);
                du -= or_conj(pv[p], om, P->eps, P->delta);
            }
        }
    *primal = pr;
    *dual = du;
}

/* ------------------------------------------------------------------------ */
/* Reverse mode of the refinement (the differentiable form): gradient of the */
/* loss mean_i |u_i - gt_i| of the refined disparity with respect to the     */
/* cost samples, the per-pixel data weights alpha_i and lambda_r.  The       */
/* labels that start the refinement are constants.  Every map of an          */
/* iteration is piecewise linear; derivatives follow the branch the forward   */
/* comparisons take (strict inequalities select the non-identity branch).    */
/* ------------------------------------------------------------------------ */

/* d interp(c, x) / dx with the argument clamp (1 inside [0, L-1], else 0) */
static double interp_dx(int L, const double* c, double u)
{
    if (u < 0.0 || u > (double)(L - 1)) return 0.0;
    double fl = floor(u);
    int k = (int)fl;
    if (k > L - 2) k = L - 2;
    return c[k + 1] - c[k];
}

/* scatter w * d interp(c, x) / dc into g */
static void interp_dc(int L, double u, double w, double* g)
{
    if (u < 0.0) u = 0.0;
    if (u > (double)(L - 1)) u = (double)(L - 1);
    double fl = floor(u);
    int k = (int)fl;
    if (k > L - 2) k = L - 2;
    if (k < 0) k = 0;
    double t = u - (double)k;
    g[k] += w * (1.0 - t);
    g[k + 1] += w * t;
}

/* forward of one prox of step * (omega r_{a,b})* with its derivatives */
static double prox_conj_d(double t, double omega, double a, double b, double step, double* dt,
                          double* domega)
{
    double tp, dtp = 1.0, dom = 0.0;
    if (fabs(t) < a * omega) {
        tp = t;
    } else {
        double m = fabs(t) - b * step;
        double s = t > 0 ? 1.0 : (t < 0 ? -1.0 : 0.0);
        if (m > a * omega) { tp = s * m; dtp = 1.0; dom = 0.0; }
        else { tp = s * a * omega; dtp = 0.0; dom = s * a; }
    }
    if (tp > omega) { tp = omega; dtp = 0.0; dom = 1.0; }
    else if (tp < -omega) { tp = -omega; dtp = 0.0; dom = -1.0; }
    *dt = dtp;
    *domega = dom;
    return tp;
}

int or_refine_grad(int H, int W, int L, const double* cost, const double* alpha, const double* wh,
                   const double* wv, const double* uinit, int iters, const or_cont_params* P,
                   const double* gt, double* u_out, double* loss, double* g_cost, double* g_alpha,
                   double* g_lambda, double* g_u0)
{
    if (H <= 0 || W <= 0 || L < 2 || P->warps <= 0 || iters < 0) return OR_ERR_ARG;
    i64 N = (i64)H * W;
    int T = iters;
    /* per-iteration input states and per-warp linearisations */
    double* U = (double*)malloc((size_t)(T + 1) * N * sizeof(double));
    double* PH = (double*)malloc((size_t)(T + 1) * N * sizeof(double));
    double* PV = (double*)malloc((size_t)(T + 1) * N * sizeof(double));
    double* QH = (double*)malloc((size_t)(T + 1) * N * sizeof(double));
    double* QV = (double*)malloc((size_t)(T + 1) * N * sizeof(double));
    int nw = P->warps;
    double* U0 = (double*)malloc((size_t)nw * N * sizeof(double));
    double* S1 = (double*)malloc((size_t)nw * N * sizeof(double));
    double* S2 = (double*)malloc((size_t)nw * N * sizeof(double));
    double* LO = (double*)malloc((size_t)nw * N * sizeof(double));
    double* HI = (double*)malloc((size_t)nw * N * sizeof(double));
    int* wstart = (int*)malloc((size_t)(nw + 1) * sizeof(int));
    const double bp = P->delta, ap = P->eps, bq = P->C + P->delta - P->eps * P->delta;
    const double tau = P->tau, sigma = P->sigma, h = P->h;
    for (i64 p = 0; p < N; ++p) { U[p] = uinit[p]; PH[p] = PV[p] = QH[p] = QV[p] = 0.0; }
    int base = T / nw, extra = T % nw, it = 0;
    for (int w = 0; w < nw; ++w) {
        wstart[w] = it;
        int nit = base + (w < extra ? 1 : 0);
        for (i64 p = 0; p < N; ++p)
            or_linearise_px(L, cost + p * L, alpha[p], U[(i64)it * N + p], h, &S1[w * N + p],
                            &S2[w * N + p], &LO[w * N + p], &HI[w * N + p]);
        for (i64 p = 0; p < N; ++p) U0[w * N + p] = U[(i64)it * N + p];
        for (int k = 0; k < nit; ++k, ++it) {
            const double *u = U + (i64)it * N, *ph = PH + (i64)it * N, *pv = PV + (i64)it * N;
            const double *qh = QH + (i64)it * N, *qv = QV + (i64)it * N;
            double *un = U + (i64)(it + 1) * N, *phn = PH + (i64)(it + 1) * N;
            double *pvn = PV + (i64)(it + 1) * N, *qhn = QH + (i64)(it + 1) * N;
            double *qvn = QV + (i64)(it + 1) * N;
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    i64 p = (i64)y * W + x;
                    double div = 0.0;
                    if (x + 1 < W) div += ph[p] - qh[p];
                    if (x > 0) div -= ph[p - 1] - qh[p - 1];
                    if (y + 1 < H) div += pv[p] - qv[p];
                    if (y > 0) div -= pv[p - W] - qv[p - W];
                    un[p] = or_prox_data(u[p] - tau * div, U0[w * N + p], S1[w * N + p], S2[w * N + p],
                                         LO[w * N + p], HI[w * N + p], tau);
                }
            for (i64 p = 0; p < N; ++p) phn[p] = pvn[p] = qhn[p] = qvn[p] = 0.0;
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    i64 p = (i64)y * W + x;
                    double d1, d2;
                    if (x + 1 < W) {
                        double om = P->lambda_r * wh[p];
                        qhn[p] = prox_conj_d(qh[p] + tau * (u[p] - u[p + 1]), om, 0.0, bq, tau, &d1, &d2);
                        phn[p] = prox_conj_d(ph[p] + sigma * ((2 * un[p] - u[p]) - (2 * un[p + 1] - u[p + 1])),
                                             om, ap, bp, sigma, &d1, &d2);
                    }
                    if (y + 1 < H) {
                        double om = P->lambda_r * wv[p];
                        qvn[p] = prox_conj_d(qv[p] + tau * (u[p] - u[p + W]), om, 0.0, bq, tau, &d1, &d2);
                        pvn[p] = prox_conj_d(pv[p] + sigma * ((2 * un[p] - u[p]) - (2 * un[p + W] - u[p + W])),
                                             om, ap, bp, sigma, &d1, &d2);
                    }
                }
        }
    }
    wstart[nw] = T;
    /* loss and its adjoint */
    const double* uT = U + (i64)T * N;
    double Ls = 0.0;
    double* ub = (double*)calloc((size_t)N, sizeof(double));   /* adjoint of u */
    double* phb = (double*)calloc((size_t)N, sizeof(double));
    double* pvb = (double*)calloc((size_t)N, sizeof(double));
    double* qhb = (double*)calloc((size_t)N, sizeof(double));
    double* qvb = (double*)calloc((size_t)N, sizeof(double));
    for (i64 p = 0; p < N; ++p) {
        double d = uT[p] - gt[p];
        Ls += fabs(d);
        ub[p] = (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) / (double)N;
        u_out[p] = uT[p];
    }
    *loss = Ls / (double)N;
    for (i64 e = 0; e < N * L; ++e) g_cost[e] = 0.0;
    for (i64 p = 0; p < N; ++p) g_alpha[p] = 0.0;
    double glam = 0.0;
    double* tqh = (double*)calloc((size_t)N, sizeof(double));
    double* tqv = (double*)calloc((size_t)N, sizeof(double));
    double* tph = (double*)calloc((size_t)N, sizeof(double));
    double* tpv = (double*)calloc((size_t)N, sizeof(double));
    double* uhb = (double*)calloc((size_t)N, sizeof(double));
    double* nub = (double*)calloc((size_t)N, sizeof(double));
    double* s1b = (double*)calloc((size_t)N, sizeof(double));
    double* s2b = (double*)calloc((size_t)N, sizeof(double));
    double* u0b = (double*)calloc((size_t)N, sizeof(double));
    double* lob = (double*)calloc((size_t)N, sizeof(double));
    double* hib = (double*)calloc((size_t)N, sizeof(double));
    for (int w = nw - 1; w >= 0; --w) {
        for (int k = wstart[w + 1] - 1; k >= wstart[w]; --k) {
            const double *u = U + (i64)k * N, *un = U + (i64)(k + 1) * N;
            const double *ph = PH + (i64)k * N, *pv = PV + (i64)k * N;
            const double *qh = QH + (i64)k * N, *qv = QV + (i64)k * N;
            /* adjoints of this iteration's outputs: ub (u+), phb.. (p+, q+) */
            for (i64 p = 0; p < N; ++p) { tqh[p] = tqv[p] = tph[p] = tpv[p] = 0.0; }
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    i64 p = (i64)y * W + x;
                    double dt, dom;
                    if (x + 1 < W) {
                        double om = P->lambda_r * wh[p];
                        prox_conj_d(qh[p] + tau * (u[p] - u[p + 1]), om, 0.0, bq, tau, &dt, &dom);
                        tqh[p] = qhb[p] * dt;
                        glam += qhb[p] * dom * wh[p];
                        prox_conj_d(ph[p] + sigma * ((2 * un[p] - u[p]) - (2 * un[p + 1] - u[p + 1])), om,
                                    ap, bp, sigma, &dt, &dom);
                        tph[p] = phb[p] * dt;
                        glam += phb[p] * dom * wh[p];
                    }
                    if (y + 1 < H) {
                        double om = P->lambda_r * wv[p];
                        prox_conj_d(qv[p] + tau * (u[p] - u[p + W]), om, 0.0, bq, tau, &dt, &dom);
                        tqv[p] = qvb[p] * dt;
                        glam += qvb[p] * dom * wv[p];
                        prox_conj_d(pv[p] + sigma * ((2 * un[p] - u[p]) - (2 * un[p + W] - u[p + W])), om,
                                    ap, bp, sigma, &dt, &dom);
                        tpv[p] = pvb[p] * dt;
                        glam += pvb[p] * dom * wv[p];
                    }
                }
            /* A^T of the edge adjoints per pixel; adjoint of u+ and of u_hat */
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    i64 p = (i64)y * W + x;
                    double atp = 0.0, atq = 0.0;
                    if (x + 1 < W) { atp += tph[p]; atq += tqh[p]; }
                    if (x > 0) { atp -= tph[p - 1]; atq -= tqh[p - 1]; }
                    if (y + 1 < H) { atp += tpv[p]; atq += tqv[p]; }
                    if (y > 0) { atp -= tpv[p - W]; atq -= tqv[p - W]; }
                    double wbar = sigma * atp;
                    double unb = ub[p] + 2.0 * wbar;       /* total adjoint of u+ */
                    nub[p] = -wbar + tau * atq;            /* direct paths into u */
                    /* reverse of the data prox and the box clamp */
                    double div = 0.0;
                    if (x + 1 < W) div += ph[p] - qh[p];
                    if (x > 0) div -= ph[p - 1] - qh[p - 1];
                    if (y + 1 < H) div += pv[p] - qv[p];
                    if (y > 0) div -= pv[p - W] - qv[p - W];
                    double uh = u[p] - tau * div;
                    double u0 = U0[w * N + p], ts1 = tau * S1[w * N + p], ts2 = tau * S2[w * N + p];
                    int cs = uh > u0 + ts2 ? 0 : (uh < u0 + ts1 ? 1 : 2);
                    double v = cs == 0 ? uh - ts2 : (cs == 1 ? uh - ts1 : u0);
                    double lo = LO[w * N + p], hi = HI[w * N + p];
                    if (v < lo) { lob[p] += unb; uhb[p] = 0.0; }
                    else if (v > hi) { hib[p] += unb; uhb[p] = 0.0; }
                    else if (cs == 0) { uhb[p] = unb; s2b[p] -= tau * unb; }
                    else if (cs == 1) { uhb[p] = unb; s1b[p] -= tau * unb; }
                    else { uhb[p] = 0.0; u0b[p] += unb; }
                }
            /* u_hat = u - tau A^T (p - q): adjoints of the inputs */
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    i64 p = (i64)y * W + x;
                    ub[p] = nub[p] + uhb[p];
                }
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    i64 p = (i64)y * W + x;
                    if (x + 1 < W) {
                        double d = uhb[p] - uhb[p + 1];
                        phb[p] = tph[p] - tau * d;
                        qhb[p] = tqh[p] + tau * d;
                    }
                    if (y + 1 < H) {
                        double d = uhb[p] - uhb[p + W];
                        pvb[p] = tpv[p] - tau * d;
                        qvb[p] = tqv[p] + tau * d;
                    }
                }
        }
        /* reverse of the linearisation at the start of warp w */
        for (i64 p = 0; p < N; ++p) {
            const double* c = cost + p * L;
            double u0 = U0[w * N + p], a = alpha[p];
            double d0 = or_interp(L, c, u0), dm = or_interp(L, c, u0 - h), dp = or_interp(L, c, u0 + h);
            double s1r = a * (d0 - dm) / h, s2r = a * (dp - d0) / h;
            double b1 = s1b[p], b2 = s2b[p];
            if (s2r < s1r) { double m = 0.5 * (b1 + b2); b1 = m; b2 = m; }
            g_alpha[p] += b1 * (d0 - dm) / h + b2 * (dp - d0) / h;
            double* gc = g_cost + p * L;
            interp_dc(L, u0, a / h * (b1 - b2), gc);
            interp_dc(L, u0 - h, -a / h * b1, gc);
            interp_dc(L, u0 + h, a / h * b2, gc);
            double gu = u0b[p];
            gu += b1 * a / h * (interp_dx(L, c, u0) - interp_dx(L, c, u0 - h));
            gu += b2 * a / h * (interp_dx(L, c, u0 + h) - interp_dx(L, c, u0));
            if (u0 - h > 0.0) gu += lob[p];
            if (u0 + h < (double)(L - 1)) gu += hib[p];
            ub[p] += gu;
            s1b[p] = s2b[p] = u0b[p] = lob[p] = hib[p] = 0.0;
        }
    }
    *g_lambda = glam;
    if (g_u0 != NULL)
        for (i64 p = 0; p < N; ++p) g_u0[p] = ub[p];
    free(U); free(PH); free(PV); free(QH); free(QV); free(U0); free(S1); free(S2); free(LO); free(HI);
    free(wstart); free(ub); free(phb); free(pvb); free(qhb); free(qvb); free(tqh); free(tqv);
    free(tph); free(tpv); free(uhb); free(nub); free(s1b); free(s2b); free(u0b); free(lob); free(hib);
    return OR_OK;
}
