/*
 * ttm_oracle.c -- plain, slow, FP64 CPU oracle for tensorial template matching
 * (Martinez-Sanchez, Homberg, Almira, Phelippeau: "Tensorial template matching
 * for fast cross-correlation with rotations and its application for
 * tomography", ECCV 2024).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call
 * this file; only the test-suite, the package's smoke check and the benchmark's
 * CPU-baseline leg do. It shares no code, header, table or helper with the
 * CUDA library: every step below is written out from the paper's definitions
 * with direct spatial sums (no FFT), in double precision, looping voxel by
 * voxel so that each line can be checked against the cited equation by eye.
 * OpenMP is used only to run independent output voxels on several cores.
 *
 * Conventions used everywhere in this file:
 *   volumes are C-order [Z][Y][X] (x fastest); a template of extent
 *   (tz,ty,tx) has its centre at (tz/2, ty/2, tx/2) and offsets
 *   p = (ix-cx, iy-cy, iz-cz); vectors are (x, y, z); quaternions are
 *   (w, x, y, z); symmetric-tensor components are the full-tensor entries
 *   indexed by multi-indices alpha in graded-lex descending order, e.g. for
 *   n = 2, d' = 3: xx, xy, xz, yy, yz, zz.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - the filter h is applied with zero padding at the volume edges;
 *   - the integral of Eq. 9 is the sample mean over Q (Alg. 1 omits 1/|Q|);
 *   - Alg. 1 (rotate t', no second S) is followed rather than Eq. 9's S(t')_R;
 *   - rotated copies are t'_R(p) = t'(R^T p), trilinear, zero outside the grid;
 *   - with d' = 3 the tensor weight of a rotation R is (R e_z)^{(x)n};
 *   - w(x) = 0 where the local variance is not above var_floor (callers use
 *     1e-8 * M * mean(g^2): below it an FP32 correlation cannot resolve the
 *     window, see the local normaliser) or not above 1e-10 * S2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_API __attribute__((visibility("default")))

static const double PI = 3.14159265358979323846264338327950288;

ORACLE_API int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

ORACLE_API void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Symmetric-tensor index set I (Alg. 1 and Alg. 2: "indices independent
 * components degree-n tensor"); |I| = binom(n + d' - 1, n) (Sec. 3).        */

ORACLE_API int oracle_num_components(int n, int d)
{
    /* binom(n + d - 1, n) by the product formula */
    long num = 1, den = 1;
    for (int i = 1; i <= n; i++) { num *= (d - 1 + i); den *= i; }
    return (int)(num / den);
}

/* Writes K rows of d exponents (alpha_1..alpha_d, summing to n), graded-lex
 * descending: the first exponent is largest first, then the second, ... */
static int fill_indices(int n, int d, int pos, int left, int* cur, int* out, int k)
{
    if (pos == d - 1) {
        cur[pos] = left;
        memcpy(out + (size_t)k * d, cur, sizeof(int) * d);
        return k + 1;
    }
    for (int e = left; e >= 0; e--) {
        cur[pos] = e;
        k = fill_indices(n, d, pos + 1, left - e, cur, out, k);
    }
    return k;
}

ORACLE_API int oracle_multi_indices(int n, int d, int* alpha)
{
    int cur[8] = {0};
    return fill_indices(n, d, 0, n, cur, alpha, 0);
}

/* multiplicity n! / prod(alpha_i!) : the number of full-tensor entries that
 * carry the value of one independent component */
static double multiplicity(const int* a, int d)
{
    int n = 0;
    for (int i = 0; i < d; i++) n += a[i];
    double v = 1.0;
    for (int i = 2; i <= n; i++) v *= i;
    for (int j = 0; j < d; j++)
        for (int i = 2; i <= a[j]; i++) v /= i;
    return v;
}

ORACLE_API void oracle_multiplicities(int n, int d, double* mult)
{
    int K = oracle_num_components(n, d);
    int* a = (int*)malloc(sizeof(int) * K * d);
    oracle_multi_indices(n, d, a);
    for (int k = 0; k < K; k++) mult[k] = multiplicity(a + k * d, d);
    free(a);
}

/* u^alpha */
static double monomial(const double* u, const int* a, int d)
{
    double v = 1.0;
    for (int i = 0; i < d; i++)
        for (int e = 0; e < a[i]; e++) v *= u[i];
    return v;
}

/* ------------------------------------------------------------------------ */
/* Eq. 3: the filter h with 1-D z-transform 1 + a(z + z^-1 - 2), i.e. taps
 * [a, 1 - 2a, a] on each axis, applied separably (as the 27-term product
 * kernel), zero outside the volume.                                          */

ORACLE_API void oracle_filter3(const double* f, int Z, int Y, int X, double a, double* g)
{
    const double tap[3] = {a, 1.0 - 2.0 * a, a};
#pragma omp parallel for schedule(static)
    for (int z = 0; z < Z; z++)
        for (int y = 0; y < Y; y++)
            for (int x = 0; x < X; x++) {
                double acc = 0.0;
                for (int dz = -1; dz <= 1; dz++)
                    for (int dy = -1; dy <= 1; dy++)
                        for (int dx = -1; dx <= 1; dx++) {
                            int zz = z + dz, yy = y + dy, xx = x + dx;
                            if (zz < 0 || zz >= Z || yy < 0 || yy >= Y || xx < 0 || xx >= X)
                                continue;
                            acc += tap[dz + 1] * tap[dy + 1] * tap[dx + 1] *
                                   f[((size_t)zz * Y + yy) * X + xx];
                        }
                g[((size_t)z * Y + y) * X + x] = acc;
            }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2 (after Eq. 2): mask m equal to 1 within radius r of the centre, 0
 * beyond a slightly larger radius r + soft, interpolated in between (here a
 * raised-cosine ramp; soft = 0 gives the binary sphere). Returns M = sum m.  */

ORACLE_API double oracle_mask(int tz, int ty, int tx, double r, double soft, double* m)
{
    int cz = tz / 2, cy = ty / 2, cx = tx / 2;
    double M = 0.0;
    for (int iz = 0; iz < tz; iz++)
        for (int iy = 0; iy < ty; iy++)
            for (int ix = 0; ix < tx; ix++) {
                double px = ix - cx, py = iy - cy, pz = iz - cz;
                double rho = sqrt(px * px + py * py + pz * pz);
                double v;
                if (rho <= r) v = 1.0;
                else if (soft > 0.0 && rho < r + soft) v = 0.5 * (1.0 + cos(PI * (rho - r) / soft));
                else v = 0.0;
                m[((size_t)iz * ty + iy) * tx + ix] = v;
                M += v;
            }
    return M;
}

/* ------------------------------------------------------------------------ */
/* Eq. 4: t' = m (S(t) - mu) / sqrt(<S(t)^2,1> - <S(t),1>^2 / M), with
 * S(t) = m (h * t) (Eq. 3), mu = (S(t) . m) / M. Returns the denominator.   */

ORACLE_API double oracle_normalise_template(const double* t, int tz, int ty, int tx,
                                            const double* m, double a, double* tp)
{
    size_t n = (size_t)tz * ty * tx;
    double* ht = (double*)malloc(sizeof(double) * n);
    oracle_filter3(t, tz, ty, tx, a, ht);
    double M = 0.0, s_dot_m = 0.0, s1 = 0.0, s2 = 0.0;
    for (size_t i = 0; i < n; i++) {
        double S = m[i] * ht[i];
        M += m[i];
        s_dot_m += S * m[i];
        s1 += S;
        s2 += S * S;
    }
    double mu = s_dot_m / M;
    double den = sqrt(s2 - s1 * s1 / M);
    for (size_t i = 0; i < n; i++) {
        double S = m[i] * ht[i];
        tp[i] = m[i] * (S - mu) / den;
    }
    free(ht);
    return den;
}

/* ------------------------------------------------------------------------ */
/* Rotations. Sec. 3 integrates over SO(3) with the uniform samples of
 * Alexa (CVPR 2022, "Super-Fibonacci spirals"): for i = 0..N-1, s = i + 1/2,
 * r = sqrt(s/N), R = sqrt(1 - s/N), alpha = 2 pi s / phi, beta = 2 pi s / psi
 * with phi = sqrt(2) and psi the real root of psi^4 = psi + 4, and the unit
 * quaternion (r sin alpha, r cos alpha, R sin beta, R cos beta), whose four
 * entries are taken here as (w, x, y, z).                                    */

static double superfib_psi(void)
{
    /* Newton on psi^4 - psi - 4 from 1.5 */
    double p = 1.5;
    for (int i = 0; i < 60; i++) p -= (p * p * p * p - p - 4.0) / (4.0 * p * p * p - 1.0);
    return p;
}

ORACLE_API double oracle_superfib_psi(void) { return superfib_psi(); }

ORACLE_API void oracle_superfib(int64_t N, double* q)
{
    const double phi = sqrt(2.0), psi = superfib_psi();
    for (int64_t i = 0; i < N; i++) {
        double s = (double)i + 0.5;
        double r = sqrt(s / (double)N), R = sqrt(1.0 - s / (double)N);
        double al = 2.0 * PI * s / phi, be = 2.0 * PI * s / psi;
        q[4 * i + 0] = r * sin(al);
        q[4 * i + 1] = r * cos(al);
        q[4 * i + 2] = R * sin(be);
        q[4 * i + 3] = R * cos(be);
    }
}

/* Hamilton product p q (so that rot(p q) = rot(p) rot(q)) */
ORACLE_API void oracle_quat_mul(const double* p, const double* q, double* o)
{
    double w = p[0] * q[0] - p[1] * q[1] - p[2] * q[2] - p[3] * q[3];
    double x = p[0] * q[1] + p[1] * q[0] + p[2] * q[3] - p[3] * q[2];
    double y = p[0] * q[2] - p[1] * q[3] + p[2] * q[0] + p[3] * q[1];
    double z = p[0] * q[3] + p[1] * q[2] - p[2] * q[1] + p[3] * q[0];
    o[0] = w; o[1] = x; o[2] = y; o[3] = z;
}

/* rotation matrix (row-major, acting on column vectors (x,y,z)) of a unit q */
ORACLE_API void oracle_quat_to_rot(const double* q, double* R)
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* The 24 proper rotations of the cube as quaternions: identity, three
 * half-turns about the axes, six quarter-turns about the axes, six
 * half-turns about face diagonals, eight third-turns about body diagonals. */
ORACLE_API void oracle_cube_rotations(double* q)
{
    const double h = sqrt(0.5);
    double list[24][4] = {
        {1, 0, 0, 0},
        {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1},
        {h, h, 0, 0}, {h, -h, 0, 0}, {h, 0, h, 0}, {h, 0, -h, 0}, {h, 0, 0, h}, {h, 0, 0, -h},
        {0, h, h, 0}, {0, h, -h, 0}, {0, h, 0, h}, {0, h, 0, -h}, {0, 0, h, h}, {0, 0, h, -h},
        {.5, .5, .5, .5}, {.5, .5, .5, -.5}, {.5, .5, -.5, .5}, {.5, .5, -.5, -.5},
        {.5, -.5, .5, .5}, {.5, -.5, .5, -.5}, {.5, -.5, -.5, .5}, {.5, -.5, -.5, -.5},
    };
    memcpy(q, list, sizeof(list));
}

/* Q = {c * q_i}: base samples q_i left-multiplied by every cube rotation c;
 * entry (i, j) is stored at row i*24 + j. Makes the quadrature exactly
 * equivariant under the cube group.                                          */
ORACLE_API void oracle_symmetrise_cube(const double* base, int64_t N, double* out)
{
    double cube[24][4];
    oracle_cube_rotations(&cube[0][0]);
    for (int64_t i = 0; i < N; i++)
        for (int j = 0; j < 24; j++) oracle_quat_mul(cube[j], base + 4 * i, out + 4 * (i * 24 + j));
}

/* ------------------------------------------------------------------------ */
/* Rotated template t'_R(p) = t'(R^{-1} p) = t'(R^T p), trilinear
 * interpolation, zero outside the template grid (reading of "rotate t'
 * according to q" in Alg. 1).                                                */

static double trilinear(const double* v, int tz, int ty, int tx, double fx, double fy, double fz)
{
    double x0 = floor(fx), y0 = floor(fy), z0 = floor(fz);
    double ax = fx - x0, ay = fy - y0, az = fz - z0;
    double acc = 0.0;
    for (int dz = 0; dz <= 1; dz++)
        for (int dy = 0; dy <= 1; dy++)
            for (int dx = 0; dx <= 1; dx++) {
                long ix = (long)x0 + dx, iy = (long)y0 + dy, iz = (long)z0 + dz;
                if (ix < 0 || ix >= tx || iy < 0 || iy >= ty || iz < 0 || iz >= tz) continue;
                double wgt = (dx ? ax : 1 - ax) * (dy ? ay : 1 - ay) * (dz ? az : 1 - az);
                acc += wgt * v[((size_t)iz * ty + iy) * tx + ix];
            }
    return acc;
}

ORACLE_API void oracle_rotate_template(const double* t, int tz, int ty, int tx, const double* q,
                                       double* out)
{
    double R[9];
    oracle_quat_to_rot(q, R);
    int cz = tz / 2, cy = ty / 2, cx = tx / 2;
    for (int iz = 0; iz < tz; iz++)
        for (int iy = 0; iy < ty; iy++)
            for (int ix = 0; ix < tx; ix++) {
                double px = ix - cx, py = iy - cy, pz = iz - cz;
                /* R^T p */
                double sx = R[0] * px + R[3] * py + R[6] * pz;
                double sy = R[1] * px + R[4] * py + R[7] * pz;
                double sz = R[2] * px + R[5] * py + R[8] * pz;
                out[((size_t)iz * ty + iy) * tx + ix] = trilinear(t, tz, ty, tx, sx + cx, sy + cy, sz + cz);
            }
}

/* ------------------------------------------------------------------------ */
/* Alg. 1 / Eq. 9: tensorial template T(t) = integral over SO(3) of
 * R^{(x)n} t'_R dR, evaluated as the mean over the samples Q. For each q the
 * rotated copy t'_q is formed, and every independent component i of the
 * tensor power receives k_i(q) t'_q, with k_i(q) = u^alpha_i for
 * u = R_q e_z (d' = 3) or u = q (d' = 4, the paper's quaternion form).
 * Output T is [K][tz][ty][tx].                                               */

ORACLE_API int oracle_tensor_field(const double* tp, int tz, int ty, int tx, const double* quats,
                                   int64_t nq, int n, int d, double* T)
{
    int K = oracle_num_components(n, d);
    int* alpha = (int*)malloc(sizeof(int) * K * d);
    oracle_multi_indices(n, d, alpha);
    size_t nv = (size_t)tz * ty * tx;
    memset(T, 0, sizeof(double) * nv * K);
    int cz = tz / 2, cy = ty / 2, cx = tx / 2;
    /* parallel over template voxels; each voxel sums over all of Q */
#pragma omp parallel for schedule(dynamic, 16)
    for (long v = 0; v < (long)nv; v++) {
        int ix = (int)(v % tx), iy = (int)((v / tx) % ty), iz = (int)(v / ((size_t)tx * ty));
        double px = ix - cx, py = iy - cy, pz = iz - cz;
        double* acc = (double*)calloc(K, sizeof(double));
        for (int64_t j = 0; j < nq; j++) {
            const double* q = quats + 4 * j;
            double R[9];
            oracle_quat_to_rot(q, R);
            double sx = R[0] * px + R[3] * py + R[6] * pz;
            double sy = R[1] * px + R[4] * py + R[7] * pz;
            double sz = R[2] * px + R[5] * py + R[8] * pz;
            double val = trilinear(tp, tz, ty, tx, sx + cx, sy + cy, sz + cz);
            if (val == 0.0) continue;
            double u[4];
            if (d == 3) { u[0] = R[2]; u[1] = R[5]; u[2] = R[8]; } /* R e_z */
            else { u[0] = q[0]; u[1] = q[1]; u[2] = q[2]; u[3] = q[3]; }
            for (int k = 0; k < K; k++) acc[k] += monomial(u, alpha + k * d, d) * val;
        }
        for (int k = 0; k < K; k++) T[(size_t)k * nv + v] = acc[k] / (double)nq;
        free(acc);
    }
    free(alpha);
    return K;
}

/* ------------------------------------------------------------------------ */
/* Eq. 2: w(x) = 1 / sqrt(<S(tau_x f)^2, 1> - <S(tau_x f), 1>^2 / M) with
 * tau_x f(z) = f(z + x) and S = m (h * .): S1 = sum_p m(p) g(x+p),
 * S2 = sum_p m(p)^2 g(x+p)^2, var = S2 - S1^2 / M, where g = h * f is the
 * filtered tomogram. The local variance is taken as zero (w = 0) where it is
 * not above var_floor or not above 1e-10 * S2, i.e. where the window is
 * constant to about five digits. The callers' var_floor, 1e-8 M mean(g^2),
 * marks windows that hold almost none of the volume's energy (a sliver of
 * an object in an empty background): there 1/sqrt(var) would amplify the
 * rounding of an FP32 correlation (about 1e-6 of its scale) past the
 * value range of an LNCC. Evaluated at the voxels listed in vox
 * (linear indices); periodic != 0 wraps x+p around the grid, otherwise
 * samples outside the volume count as 0.                                     */

static inline int wrap_or_out(long v, long n, int periodic, long* o)
{
    if (v >= 0 && v < n) { *o = v; return 1; }
    if (!periodic) return 0;
    v %= n;
    if (v < 0) v += n;
    *o = v;
    return 1;
}

ORACLE_API double oracle_global_variance(const double* g, int64_t n)
{
    double s = 0.0, s2 = 0.0;
    for (int64_t i = 0; i < n; i++) { s += g[i]; s2 += g[i] * g[i]; }
    double mean = s / (double)n;
    return s2 / (double)n - mean * mean;
}

ORACLE_API double oracle_mean_square(const double* g, int64_t n)
{
    double s2 = 0.0;
    for (int64_t i = 0; i < n; i++) s2 += g[i] * g[i];
    return s2 / (double)n;
}

ORACLE_API void oracle_local_w(const double* g, int Z, int Y, int X, const double* m, int tz, int ty,
                               int tx, int periodic, double var_floor, const int64_t* vox,
                               int64_t nvox, double* w, double* S1out, double* S2out)
{
    int cz = tz / 2, cy = ty / 2, cx = tx / 2;
    double M = 0.0;
    for (size_t i = 0; i < (size_t)tz * ty * tx; i++) M += m[i];
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < nvox; i++) {
        long v = (long)vox[i];
        long x = v % X, y = (v / X) % Y, z = v / ((long)X * Y);
        double S1 = 0.0, S2 = 0.0;
        for (int iz = 0; iz < tz; iz++)
            for (int iy = 0; iy < ty; iy++)
                for (int ix = 0; ix < tx; ix++) {
                    double mv = m[((size_t)iz * ty + iy) * tx + ix];
                    if (mv == 0.0) continue;
                    long zz, yy, xx;
                    if (!wrap_or_out(z + iz - cz, Z, periodic, &zz)) continue;
                    if (!wrap_or_out(y + iy - cy, Y, periodic, &yy)) continue;
                    if (!wrap_or_out(x + ix - cx, X, periodic, &xx)) continue;
                    double gv = g[((size_t)zz * Y + yy) * X + xx];
                    S1 += mv * gv;
                    S2 += mv * mv * gv * gv;
                }
        double var = S2 - S1 * S1 / M;
        w[i] = (var > var_floor && var > 1e-10 * S2) ? 1.0 / sqrt(var) : 0.0;
        if (S1out) S1out[i] = S1;
        if (S2out) S2out[i] = S2;
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. 5 / Eq. 8 / Alg. 2: C_i(x) = w(x) (g * T_i)(x) with the correlation
 * (g * T)(x) = sum_p g(x + p) T(p), by direct summation (no FFT), for all K
 * components at the listed voxels. Output C is [K][nvox]; pass w = NULL for
 * the unnormalised correlation.                                              */

ORACLE_API void oracle_correlate(const double* g, int Z, int Y, int X, const double* T, int K,
                                 int tz, int ty, int tx, int periodic, const int64_t* vox,
                                 int64_t nvox, const double* w, double* C)
{
    int cz = tz / 2, cy = ty / 2, cx = tx / 2;
    size_t nv = (size_t)tz * ty * tx;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nvox; i++) {
        long v = (long)vox[i];
        long x = v % X, y = (v / X) % Y, z = v / ((long)X * Y);
        double* acc = (double*)calloc(K, sizeof(double));
        for (int iz = 0; iz < tz; iz++)
            for (int iy = 0; iy < ty; iy++)
                for (int ix = 0; ix < tx; ix++) {
                    long zz, yy, xx;
                    if (!wrap_or_out(z + iz - cz, Z, periodic, &zz)) continue;
                    if (!wrap_or_out(y + iy - cy, Y, periodic, &yy)) continue;
                    if (!wrap_or_out(x + ix - cx, X, periodic, &xx)) continue;
                    double gv = g[((size_t)zz * Y + yy) * X + xx];
                    size_t p = ((size_t)iz * ty + iy) * tx + ix;
                    for (int k = 0; k < K; k++) acc[k] += gv * T[(size_t)k * nv + p];
                }
        double s = w ? w[i] : 1.0;
        for (int k = 0; k < K; k++) C[(size_t)k * nvox + i] = s * acc[k];
        free(acc);
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2: scalar map c_n(x) = ||C_n(x)||_F. With C stored by independent
 * components, ||C||_F^2 = sum_alpha mult(alpha) C_alpha^2.                   */

ORACLE_API void oracle_frobenius(const double* C, int K, int n, int d, int64_t nvox, double* F)
{
    double* mult = (double*)malloc(sizeof(double) * K);
    oracle_multiplicities(n, d, mult);
    for (int64_t i = 0; i < nvox; i++) {
        double s = 0.0;
        for (int k = 0; k < K; k++) s += mult[k] * C[(size_t)k * nvox + i] * C[(size_t)k * nvox + i];
        F[i] = sqrt(s);
    }
    free(mult);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1: the orientation is the maximiser of the form
 * p(u) = C . u^{(x)n} = sum_alpha mult(alpha) C_alpha u^alpha over unit u
 * (the dominant Z-eigenpair). The oracle takes the global maximum by dense
 * sampling of the half-sphere (p is even for even n), takes the best 8
 * discrete local maxima of the sampled values as starts, and polishes each
 * to a local maximum: shifted symmetric
 * higher-order power steps (Kolda & Mayo 2011) with shift (n-1)||C||_F, which
 * never decrease p, and Riemannian Newton steps on the sphere that are kept
 * only when they do not decrease p. Gradient and Hessian are the
 * derivatives of the polynomial itself.                                      */

typedef struct {
    int n, d, K;
    const int* alpha;
    const double* mult;
} poly_t;

/* u_i^e with the convention u^0 = 1 (also for u_i = 0) */
static double ipow(double x, int e)
{
    double v = 1.0;
    for (int i = 0; i < e; i++) v *= x;
    return v;
}

static void poly_eval(const poly_t* P, const double* C, const double* u, double* pval, double* grad,
                      double* hess)
{
    int d = P->d;
    double p = 0.0;
    double gr[4] = {0, 0, 0, 0};
    double H[16] = {0};
    for (int k = 0; k < P->K; k++) {
        const int* a = P->alpha + k * d;
        double c = P->mult[k] * C[k];
        p += c * monomial(u, a, d);
        if (!grad) continue;
        for (int i = 0; i < d; i++) {
            if (a[i] == 0) continue;
            double t = c * a[i] * ipow(u[i], a[i] - 1);
            for (int j = 0; j < d; j++) if (j != i) t *= ipow(u[j], a[j]);
            gr[i] += t;
        }
        if (!hess) continue;
        for (int i = 0; i < d; i++)
            for (int j = 0; j < d; j++) {
                double t;
                if (i == j) {
                    if (a[i] < 2) continue;
                    t = c * a[i] * (a[i] - 1) * ipow(u[i], a[i] - 2);
                    for (int l = 0; l < d; l++) if (l != i) t *= ipow(u[l], a[l]);
                } else {
                    if (a[i] < 1 || a[j] < 1) continue;
                    t = c * a[i] * a[j] * ipow(u[i], a[i] - 1) * ipow(u[j], a[j] - 1);
                    for (int l = 0; l < d; l++) if (l != i && l != j) t *= ipow(u[l], a[l]);
                }
                H[i * d + j] += t;
            }
    }
    *pval = p;
    if (grad) memcpy(grad, gr, sizeof(double) * d);
    if (hess) memcpy(hess, H, sizeof(double) * d * d);
}

static void normalise(double* u, int d)
{
    double s = 0.0;
    for (int i = 0; i < d; i++) s += u[i] * u[i];
    s = sqrt(s);
    for (int i = 0; i < d; i++) u[i] /= s;
}

/* orthonormal basis of the tangent space u^perp (d-1 vectors of length d):
 * the Householder reflection H = I - 2 v v^T / (v^T v), v = u + sign(u_k) e_k
 * with k the largest entry of u, maps e_k to -sign(u_k) u, so its other
 * columns are orthonormal and orthogonal to u. */
static void tangent_basis(const double* u, int d, double* B)
{
    int k = 0;
    for (int i = 1; i < d; i++) if (fabs(u[i]) > fabs(u[k])) k = i;
    double v[4];
    for (int i = 0; i < d; i++) v[i] = u[i];
    v[k] += u[k] >= 0 ? 1.0 : -1.0;
    double vv = 0.0;
    for (int i = 0; i < d; i++) vv += v[i] * v[i];
    int got = 0;
    for (int j = 0; j < d; j++) {
        if (j == k) continue;
        for (int i = 0; i < d; i++) B[got * d + i] = (i == j ? 1.0 : 0.0) - 2.0 * v[i] * v[j] / vv;
        got++;
    }
}

/* Cholesky solve of A x = b for a small symmetric positive definite A (m x m);
 * returns 0 if A is not positive definite */
static int chol_solve(double* A, int m, const double* b, double* x)
{
    double L[9] = {0};
    for (int i = 0; i < m; i++)
        for (int j = 0; j <= i; j++) {
            double s = A[i * m + j];
            for (int k = 0; k < j; k++) s -= L[i * m + k] * L[j * m + k];
            if (i == j) {
                if (s <= 0.0) return 0;
                L[i * m + i] = sqrt(s);
            } else {
                L[i * m + j] = s / L[j * m + j];
            }
        }
    double y[3];
    for (int i = 0; i < m; i++) {
        double s = b[i];
        for (int k = 0; k < i; k++) s -= L[i * m + k] * y[k];
        y[i] = s / L[i * m + i];
    }
    for (int i = m - 1; i >= 0; i--) {
        double s = y[i];
        for (int k = i + 1; k < m; k++) s -= L[k * m + i] * x[k];
        x[i] = s / L[i * m + i];
    }
    return 1;
}

/* Polish u (in place) to a local maximum of p; returns p(u). */
static double polish(const poly_t* P, const double* C, double frob, double* u, int* iters_out)
{
    int d = P->d, n = P->n;
    double shift = (n - 1) * frob; /* bounds the spectral radius of the Hessian term */
    double p, gr[4], H[16], B[12];
    int it;
    for (it = 0; it < 400; it++) {
        poly_eval(P, C, u, &p, gr, H);
        tangent_basis(u, d, B);
        double ug = 0.0;
        for (int i = 0; i < d; i++) ug += u[i] * gr[i];
        /* Riemannian gradient and Hessian in the tangent basis */
        double g_r[3], negH[9];
        double gnorm = 0.0;
        for (int a = 0; a < d - 1; a++) {
            double s = 0.0;
            for (int i = 0; i < d; i++) s += B[a * d + i] * gr[i];
            g_r[a] = s;
            gnorm += s * s;
        }
        gnorm = sqrt(gnorm);
        if (gnorm <= 1e-13 * (frob > 1e-300 ? frob : 1.0)) break;
        for (int a = 0; a < d - 1; a++)
            for (int b = 0; b < d - 1; b++) {
                double s = 0.0;
                for (int i = 0; i < d; i++)
                    for (int j = 0; j < d; j++) s += B[a * d + i] * H[i * d + j] * B[b * d + j];
                if (a == b) s -= ug;
                negH[a * (d - 1) + b] = -s;
            }
        double xi[3];
        int took_newton = 0;
        if (chol_solve(negH, d - 1, g_r, xi)) {
            double ut[4];
            for (int i = 0; i < d; i++) {
                ut[i] = u[i];
                for (int a = 0; a < d - 1; a++) ut[i] += B[a * d + i] * xi[a];
            }
            normalise(ut, d);
            double pt;
            poly_eval(P, C, ut, &pt, NULL, NULL);
            if (pt >= p - 1e-15 * (frob > 0 ? frob : 1.0)) {
                memcpy(u, ut, sizeof(double) * d);
                took_newton = 1;
            }
        }
        if (!took_newton) {
            /* SS-HOPM step: u <- normalise(grad/n + shift u) */
            for (int i = 0; i < d; i++) u[i] = gr[i] / n + shift * u[i];
            normalise(u, d);
        }
    }
    poly_eval(P, C, u, &p, NULL, NULL);
    if (iters_out) *iters_out = it;
    return p;
}

/* Canonical representative of +-u: the last non-zero coordinate (z for
 * d' = 3) positive; for d' = 4 the first (w) non-negative, i.e. the
 * convention q ~ -q. Entries are checked in the order (z, y, x) for d' = 3
 * and (w, x, y, z) for d' = 4.                                               */
static void canonicalise(double* u, int d)
{
    int order3[3] = {2, 1, 0}, order4[4] = {0, 1, 2, 3};
    int* ord = d == 3 ? order3 : order4;
    for (int t = 0; t < d; t++) {
        double v = u[ord[t]];
        if (v > 0) return;
        if (v < 0) {
            for (int i = 0; i < d; i++) u[i] = -u[i];
            return;
        }
    }
}

/* half-sphere sample directions: spherical Fibonacci on S^2 (z > 0), or
 * super-Fibonacci quaternions on S^3 */
ORACLE_API void oracle_sample_directions(int d, int ns, double* U)
{
    if (d == 3) {
        const double ga = PI * (3.0 - sqrt(5.0)); /* golden angle */
        for (int i = 0; i < ns; i++) {
            double z = ((double)i + 0.5) / ns;
            double rr = sqrt(1.0 - z * z);
            double ph = ga * i;
            U[3 * i + 0] = rr * cos(ph);
            U[3 * i + 1] = rr * sin(ph);
            U[3 * i + 2] = z;
        }
    } else {
        oracle_superfib(ns, U);
    }
}

#define NNB 8

/* smallest eigenvalue of a small symmetric matrix (m <= 3) by cyclic Jacobi
 * rotations */
static double min_eig_sym(double* A, int m)
{
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0.0;
        for (int p = 0; p < m; p++)
            for (int q = p + 1; q < m; q++) off += A[p * m + q] * A[p * m + q];
        if (off < 1e-30) break;
        for (int p = 0; p < m; p++)
            for (int q = p + 1; q < m; q++) {
                double apq = A[p * m + q];
                if (fabs(apq) < 1e-300) continue;
                double th = 0.5 * atan2(2.0 * apq, A[q * m + q] - A[p * m + p]);
                double c = cos(th), sn = sin(th);
                for (int k = 0; k < m; k++) {
                    double akp = A[k * m + p], akq = A[k * m + q];
                    A[k * m + p] = c * akp - sn * akq;
                    A[k * m + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < m; k++) {
                    double apk = A[p * m + k], aqk = A[q * m + k];
                    A[p * m + k] = c * apk - sn * aqk;
                    A[q * m + k] = sn * apk + c * aqk;
                }
            }
    }
    double mn = A[0];
    for (int i = 1; i < m; i++) if (A[i * m + i] < mn) mn = A[i * m + i];
    return mn;
}

/* curvature of p at a maximiser u: the smallest eigenvalue of minus the
 * Riemannian Hessian (tangent space) -- how sharply the maximum is defined */
static double curvature_at(const poly_t* P, const double* C, const double* u)
{
    int d = P->d;
    double p, gr[4], H[16], B[12], A[9];
    poly_eval(P, C, u, &p, gr, H);
    tangent_basis(u, d, B);
    double ug = 0.0;
    for (int i = 0; i < d; i++) ug += u[i] * gr[i];
    for (int a = 0; a < d - 1; a++)
        for (int b = 0; b < d - 1; b++) {
            double s = 0.0;
            for (int i = 0; i < d; i++)
                for (int j = 0; j < d; j++) s += B[a * d + i] * H[i * d + j] * B[b * d + j];
            if (a == b) s -= ug;
            A[a * (d - 1) + b] = -s;
        }
    return min_eig_sym(A, d - 1);
}

/* For each voxel i: s[i] = max p, u[i*d..] = canonical argmax,
 * second[i] = the best value of a local maximum at least 1 degree away from
 * the argmax (or -inf), curv[i] (if not NULL) = curvature at the argmax.     */
ORACLE_API void oracle_maximise(const double* C, int64_t nvox, int n, int d, int nsamples,
                                double* s, double* u, double* second, double* curv)
{
    int K = oracle_num_components(n, d);
    int* alpha = (int*)malloc(sizeof(int) * K * d);
    double* mult = (double*)malloc(sizeof(double) * K);
    oracle_multi_indices(n, d, alpha);
    oracle_multiplicities(n, d, mult);
    double* U = (double*)malloc(sizeof(double) * d * nsamples);
    oracle_sample_directions(d, nsamples, U);
    /* Phi[j][k] = mult_k U_j^alpha_k so that p(U_j) = sum_k Phi[j][k] C_k */
    double* Phi = (double*)malloc(sizeof(double) * (size_t)nsamples * K);
    for (int j = 0; j < nsamples; j++)
        for (int k = 0; k < K; k++) Phi[(size_t)j * K + k] = mult[k] * monomial(U + j * d, alpha + k * d, d);
    poly_t P = {n, d, K, alpha, mult};
    const double cos1 = cos(1.0 * PI / 180.0);
    /* the NNB nearest samples of every sample, with u and -u identified
     * (closeness = |u_i . u_j|) */
    int* nbr = (int*)malloc(sizeof(int) * (size_t)nsamples * NNB);
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < nsamples; i++) {
        double bd[NNB];
        int bi[NNB], nb = 0;
        for (int j = 0; j < nsamples; j++) {
            if (j == i) continue;
            double dot = 0.0;
            for (int e = 0; e < d; e++) dot += U[i * d + e] * U[j * d + e];
            dot = fabs(dot);
            if (nb == NNB && dot <= bd[NNB - 1]) continue;
            int pos = nb < NNB ? nb++ : NNB - 1;
            while (pos > 0 && bd[pos - 1] < dot) { bd[pos] = bd[pos - 1]; bi[pos] = bi[pos - 1]; pos--; }
            bd[pos] = dot;
            bi[pos] = j;
        }
        for (int b = 0; b < NNB; b++) nbr[(size_t)i * NNB + b] = b < nb ? bi[b] : i;
    }
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t v = 0; v < nvox; v++) {
        double c[128];
        double frob2 = 0.0;
        for (int k = 0; k < K; k++) {
            c[k] = C[(size_t)k * nvox + v];
            frob2 += mult[k] * c[k] * c[k];
        }
        double frob = sqrt(frob2);
        double* pv = (double*)malloc(sizeof(double) * nsamples);
        for (int j = 0; j < nsamples; j++) {
            double acc = 0.0;
            for (int k = 0; k < K; k++) acc += Phi[(size_t)j * K + k] * c[k];
            pv[j] = acc;
        }
        /* starts: the samples that are not below any of their NNB nearest
         * samples (discrete local maxima), best first, at most 8 */
        int starts[8], ns = 0;
        for (int j = 0; j < nsamples; j++) {
            int is_max = 1;
            for (int b = 0; b < NNB && is_max; b++) if (pv[nbr[(size_t)j * NNB + b]] > pv[j]) is_max = 0;
            if (!is_max) continue;
            /* insert j into the list kept in decreasing value (index on ties) */
            int pos = ns;
            while (pos > 0 && pv[starts[pos - 1]] < pv[j]) pos--;
            if (pos >= 8) continue;
            for (int t = (ns < 8 ? ns : 7); t > pos; t--) starts[t] = starts[t - 1];
            starts[pos] = j;
            if (ns < 8) ns++;
        }
        double best = -INFINITY, sec = -INFINITY, ub[4] = {0, 0, 0, 0};
        double found_u[8][4], found_p[8];
        for (int t = 0; t < ns; t++) {
            double uu[4];
            memcpy(uu, U + starts[t] * d, sizeof(double) * d);
            found_p[t] = polish(&P, c, frob, uu, NULL);
            memcpy(found_u[t], uu, sizeof(double) * d);
            if (found_p[t] > best) { best = found_p[t]; memcpy(ub, uu, sizeof(double) * d); }
        }
        for (int t = 0; t < ns; t++) {
            double dot = 0.0;
            for (int i = 0; i < d; i++) dot += found_u[t][i] * ub[i];
            if (fabs(dot) < cos1 && found_p[t] > sec) sec = found_p[t];
        }
        if (curv) curv[v] = curvature_at(&P, c, ub);
        canonicalise(ub, d);
        s[v] = best;
        for (int i = 0; i < d; i++) u[(size_t)v * d + i] = ub[i];
        if (second) second[v] = sec;
        free(pv);
    }
    free(alpha); free(mult); free(U); free(Phi); free(nbr);
}

/* Polynomial value, Euclidean gradient and Hessian at u (exposed for the
 * eigen-residual pins). grad has d entries, hess d*d.                        */
ORACLE_API double oracle_poly_eval(const double* C, int n, int d, const double* u, double* grad,
                                   double* hess)
{
    int K = oracle_num_components(n, d);
    int* alpha = (int*)malloc(sizeof(int) * K * d);
    double* mult = (double*)malloc(sizeof(double) * K);
    oracle_multi_indices(n, d, alpha);
    oracle_multiplicities(n, d, mult);
    poly_t P = {n, d, K, alpha, mult};
    double p;
    poly_eval(&P, C, u, &p, grad, hess);
    free(alpha); free(mult);
    return p;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.4 "Find Peaks": the P highest values with a minimum exclusion
 * distance between accepted peaks. Candidates are the voxels of the box
 * [z0,z1) x [y0,y1) x [x0,x1) that beat every 26-neighbour inside the box
 * (higher value, or equal value and lower linear index); they are taken in
 * order (value descending, index ascending) and accepted when their
 * Euclidean distance to every accepted peak is at least min_dist.
 * Returns the number of peaks written.                                       */

typedef struct { double v; int64_t i; } pk_t;
static int cmp_pk(const void* a, const void* b)
{
    const pk_t* x = (const pk_t*)a;
    const pk_t* y = (const pk_t*)b;
    if (x->v > y->v) return -1;
    if (x->v < y->v) return 1;
    return x->i < y->i ? -1 : (x->i > y->i);
}

ORACLE_API int oracle_find_peaks(const double* s, int Z, int Y, int X, int z0, int z1, int y0, int y1,
                                 int x0, int x1, int P, double min_dist, int64_t* idx, double* val)
{
    size_t cap = 1024, nc = 0;
    pk_t* cand = (pk_t*)malloc(sizeof(pk_t) * cap);
    for (int z = z0; z < z1; z++)
        for (int y = y0; y < y1; y++)
            for (int x = x0; x < x1; x++) {
                int64_t i = ((int64_t)z * Y + y) * X + x;
                double v = s[i];
                int is_max = 1;
                for (int dz = -1; dz <= 1 && is_max; dz++)
                    for (int dy = -1; dy <= 1 && is_max; dy++)
                        for (int dx = -1; dx <= 1 && is_max; dx++) {
                            if (!dz && !dy && !dx) continue;
                            int zz = z + dz, yy = y + dy, xx = x + dx;
                            if (zz < z0 || zz >= z1 || yy < y0 || yy >= y1 || xx < x0 || xx >= x1)
                                continue;
                            int64_t j = ((int64_t)zz * Y + yy) * X + xx;
                            double o = s[j];
                            if (o > v || (o == v && j < i)) is_max = 0;
                        }
                if (!is_max) continue;
                if (nc == cap) { cap *= 2; cand = (pk_t*)realloc(cand, sizeof(pk_t) * cap); }
                cand[nc].v = v;
                cand[nc].i = i;
                nc++;
            }
    qsort(cand, nc, sizeof(pk_t), cmp_pk);
    int got = 0;
    double md2 = min_dist * min_dist;
    for (size_t c = 0; c < nc && got < P; c++) {
        int64_t i = cand[c].i;
        double x = (double)(i % X), y = (double)((i / X) % Y), z = (double)(i / ((int64_t)X * Y));
        int ok = 1;
        for (int a = 0; a < got && ok; a++) {
            int64_t j = idx[a];
            double xa = (double)(j % X), ya = (double)((j / X) % Y), za = (double)(j / ((int64_t)X * Y));
            double d2 = (x - xa) * (x - xa) + (y - ya) * (y - ya) + (z - za) * (z - za);
            if (d2 < md2) ok = 0;
        }
        if (!ok) continue;
        idx[got] = i;
        val[got] = cand[c].v;
        got++;
    }
    free(cand);
    return got;
}

/* ------------------------------------------------------------------------ */
/* Classical template matching, Eqs. 1, 6, 7: c(x, R) = w(x) (g * t'_R)(x) for
 * every rotation in the list (taken in list order), keeping the maximum and
 * the index of the first rotation that attains it.                           */

ORACLE_API void oracle_tm(const double* g, int Z, int Y, int X, const double* tp, int tz, int ty,
                          int tx, const double* quats, int64_t nq, int periodic, const int64_t* vox,
                          int64_t nvox, const double* w, double* best, int32_t* best_idx)
{
    size_t nv = (size_t)tz * ty * tx;
    double* rot = (double*)malloc(sizeof(double) * nv);
    double* c = (double*)malloc(sizeof(double) * nvox);
    for (int64_t i = 0; i < nvox; i++) { best[i] = -INFINITY; best_idx[i] = -1; }
    for (int64_t j = 0; j < nq; j++) {
        oracle_rotate_template(tp, tz, ty, tx, quats + 4 * j, rot);
        oracle_correlate(g, Z, Y, X, rot, 1, tz, ty, tx, periodic, vox, nvox, w, c);
        for (int64_t i = 0; i < nvox; i++)
            if (c[i] > best[i]) { best[i] = c[i]; best_idx[i] = (int32_t)j; }
    }
    free(rot);
    free(c);
}

/* ------------------------------------------------------------------------ */
/* Learned warm start (reference for the GPU training and inference): an MLP
 * K -> H -> H -> 3 with GELU activations in their tanh form,
 * GELU(x) = x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))) / 2,
 * whose output y is normalised, u_hat = y/|y|,
 * to predict the maximising direction of p_x from the components scaled to
 * unit Frobenius norm. Loss per sample: 1 - (u_hat . u*)^2, which does not
 * depend on the sign of u* (the maximiser is defined up to sign).
 * Parameters, flat: W1 [H][K], b1 [H], W2 [H][H], b2 [H], W3 [3][H], b3 [3]. */

static double gelu(double x)
{
    const double c = sqrt(2.0 / PI);
    return 0.5 * x * (1.0 + tanh(c * (x + 0.044715 * x * x * x)));
}
/* derivative of the tanh form: with t = tanh(c (x + 0.044715 x^3)),
 * GELU'(x) = (1 + t)/2 + x (1 - t^2) c (1 + 3 * 0.044715 x^2) / 2 */
static double gelu_grad(double x)
{
    const double c = sqrt(2.0 / PI);
    const double t = tanh(c * (x + 0.044715 * x * x * x));
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * c * (1.0 + 3.0 * 0.044715 * x * x);
}

ORACLE_API int64_t oracle_mlp_num_params(int K, int H) { return (int64_t)H * K + H + H * H + H + 3 * H + 3; }

/* forward for n samples; out = u_hat [n][3]; loss (sum over samples) if
 * U != NULL; grad (sum over samples, same layout as params) if grad != NULL */
ORACLE_API double oracle_mlp(const double* params, int K, int H, const double* X, const double* U, int64_t n,
                             double* out, double* grad)
{
    const double* W1 = params;
    const double* b1 = W1 + (size_t)H * K;
    const double* W2 = b1 + H;
    const double* b2 = W2 + (size_t)H * H;
    const double* W3 = b2 + H;
    const double* b3 = W3 + 3 * H;
    double *gW1 = NULL, *gb1 = NULL, *gW2 = NULL, *gb2 = NULL, *gW3 = NULL, *gb3 = NULL;
    if (grad) {
        memset(grad, 0, sizeof(double) * oracle_mlp_num_params(K, H));
        gW1 = grad; gb1 = gW1 + (size_t)H * K; gW2 = gb1 + H; gb2 = gW2 + (size_t)H * H; gW3 = gb2 + H; gb3 = gW3 + 3 * H;
    }
    double* a1 = (double*)malloc(sizeof(double) * H);
    double* h1 = (double*)malloc(sizeof(double) * H);
    double* a2 = (double*)malloc(sizeof(double) * H);
    double* h2 = (double*)malloc(sizeof(double) * H);
    double* d2 = (double*)malloc(sizeof(double) * H);
    double* d1 = (double*)malloc(sizeof(double) * H);
    double loss = 0.0;
    for (int64_t s = 0; s < n; s++) {
        const double* x = X + (size_t)s * K;
        for (int i = 0; i < H; i++) {
            double acc = b1[i];
            for (int k = 0; k < K; k++) acc += W1[(size_t)i * K + k] * x[k];
            a1[i] = acc;
            h1[i] = gelu(acc);
        }
        for (int i = 0; i < H; i++) {
            double acc = b2[i];
            for (int k = 0; k < H; k++) acc += W2[(size_t)i * H + k] * h1[k];
            a2[i] = acc;
            h2[i] = gelu(acc);
        }
        double y[3];
        for (int c = 0; c < 3; c++) {
            double acc = b3[c];
            for (int k = 0; k < H; k++) acc += W3[(size_t)c * H + k] * h2[k];
            y[c] = acc;
        }
        double ny = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
        double uh[3] = {y[0] / ny, y[1] / ny, y[2] / ny};
        if (out) for (int c = 0; c < 3; c++) out[(size_t)s * 3 + c] = uh[c];
        if (!U) continue;
        const double* us = U + (size_t)s * 3;
        double dot = uh[0] * us[0] + uh[1] * us[1] + uh[2] * us[2];
        loss += 1.0 - dot * dot;
        if (!grad) continue;
        /* dL/du_hat = -2 dot u*; dL/dy = (I - u_hat u_hat^T) dL/du_hat / |y| */
        double gu[3] = {-2.0 * dot * us[0], -2.0 * dot * us[1], -2.0 * dot * us[2]};
        double ug = uh[0] * gu[0] + uh[1] * gu[1] + uh[2] * gu[2];
        double gy[3];
        for (int c = 0; c < 3; c++) gy[c] = (gu[c] - ug * uh[c]) / ny;
        for (int c = 0; c < 3; c++) {
            gb3[c] += gy[c];
            for (int k = 0; k < H; k++) gW3[(size_t)c * H + k] += gy[c] * h2[k];
        }
        for (int k = 0; k < H; k++) {
            double g = 0.0;
            for (int c = 0; c < 3; c++) g += W3[(size_t)c * H + k] * gy[c];
            d2[k] = g * gelu_grad(a2[k]);
        }
        for (int i = 0; i < H; i++) {
            gb2[i] += d2[i];
            for (int k = 0; k < H; k++) gW2[(size_t)i * H + k] += d2[i] * h1[k];
        }
        for (int k = 0; k < H; k++) {
            double g = 0.0;
            for (int i = 0; i < H; i++) g += W2[(size_t)i * H + k] * d2[i];
            d1[k] = g * gelu_grad(a1[k]);
        }
        for (int i = 0; i < H; i++) {
            gb1[i] += d1[i];
            for (int k = 0; k < K; k++) gW1[(size_t)i * K + k] += d1[i] * x[k];
        }
    }
    free(a1); free(h1); free(a2); free(h2); free(d2); free(d1);
    return loss;
}
