// ttm_peakmap4.cu -- the quaternion form of the score (d' = 4, Sec. 3 and
// Sec. 3.1): per voxel
//   s(x) = max_{|q|=1} p_x(q),  q*(x) = argmax,
//   p_x(q) = C(x) . q^{(x)n} = sum_alpha mult(alpha) C_alpha(x) q^alpha,
// over unit quaternions q = (w, x, y, z). p is even (n even) and q, -q are
// the same rotation, so q* is reported with its first non-zero entry
// positive. The maximiser returns a full rotation, roll included.
//
// Design (one thread per voxel, components loaded structure-of-arrays):
//  * probes: 512 super-Fibonacci quaternions on the half-sphere w >= 0,
//    grouped on the host into 64 cells of 8 neighbouring probes (greedy
//    nearest-neighbour clusters); the table rows are permuted so that the
//    8 probes of a cell are exactly the columns one lane of a warp holds
//    in four consecutive 8-column tiles of the tensor-core product, so a
//    cell's best needs no shuffle;
//  * probe values p_j / ||C||_F of a warp's 32 voxels come from m16n8k16
//    FP16 products (x = C / ||C||_F, weighted monomials), FP32 accumulate;
//    only the best probe of each cell is kept, as a 16-bit key (order-
//    preserving FP16 bits with the probe's place in the cell in the low 3
//    bits), in shared memory [cell][thread];
//  * starts by angular suppression over the cell bests: the best probe,
//    then the best cell best farther than 25 degrees (|q . q_s| <
//    cos 25 deg) from every start taken, if within 0.2 ||C||_F (n = 4) or
//    0.5 ||C||_F (n = 6) of the best, up to 4 (n = 4) or 6 (n = 6) starts;
//  * n = 2 needs no probes: p = q^T A q with A_ij = C_{e_i + e_j}, whose
//    maximum over unit q is the top eigenpair of the symmetric 4 x 4
//    matrix A (cyclic Jacobi rotations), polished by Newton;
//  * up to three Riemannian Newton steps from every start in turn (one copy
//    of the step code, so the kernel stays small in the instruction cache),
//    then up to twelve on the best. S^3 is parallelisable: q (x) i,
//    q (x) j, q (x) k (quaternion products) are an orthonormal basis of the
//    tangent space at q, so no Householder branch is needed. The
//    derivatives come from the contraction A = C . q^{n-2} (a symmetric
//    4 x 4 matrix): p = q^T A q, grad p = n A q, Hess p = n (n-1) A. Minus
//    the Riemannian Hessian is factored by LDL^T; where it is not positive
//    definite it is shifted by its smallest eigenvalue (closed form for
//    symmetric 3 x 3, Smith 1961) to 0.05 ||C||_F (a Levenberg-Marquardt
//    step); steps are limited to 0.2 rad and halved until p does not
//    decrease, and a shifted power step (SS-HOPM, shift (n-1) ||C||_F) is
//    the last resort.
// The probe count, cell size, separation and step counts were chosen by an
// emulation against the FP64 maximiser on random and on correlation-derived
// tensors (0 to 1 misses in 20 000 random tensors).
#include <algorithm>
#include <cmath>
#include <vector>

#include <cuda_fp16.h>

#include "mlp_mma.cuh"
#include "ttm_internal.h"

namespace ttm {

constexpr int kP4 = 512;                 // probes on the half 3-sphere
constexpr int kP4Cells = kP4 / 8;        // one cell per 8-column MMA tile
constexpr int kP4Threads = 256;
constexpr int kP4Pre = 3;                // Newton steps per start (starts in turn)
constexpr int kP4Polish = 12;            // Newton steps on the best start
constexpr float kP4SepCos = 0.90630779f; // starts lie farther apart than 25 degrees

__host__ __device__ constexpr int ncomp4(int n) { return (n + 1) * (n + 2) * (n + 3) / 6; }
// Starts within this * ||C||_F of the best probe. The drop of the form from
// a maximum to the nearest probe is at most half the Hessian bound
// n (n - 1) ||C||_F times the squared probe spacing, so the margin scales
// with n (n - 1): 0.2 at n = 4 (chosen by emulation against the oracle),
// 0.5 at n = 6.
__host__ __device__ constexpr float p4_margin(int n) { return n >= 6 ? 0.5f : 0.2f; }
__host__ __device__ constexpr int nstarts4(int n) { return n >= 6 ? 6 : (n >= 4 ? 4 : 2); }
__host__ __device__ constexpr int p4_kx(int n) { return (ncomp4(n) + 15) / 16 * 16; }
__host__ __device__ constexpr int p4_kxs(int n) { return p4_kx(n) + 8; }
__host__ __device__ constexpr int p4_kp(int n) { return (ncomp4(n) + 3) / 4 * 4; }
__host__ __device__ constexpr float fact4(int n) { return n <= 1 ? 1.f : n * fact4(n - 1); }

// position of exponents (a, b, c, n-a-b-c) of (w, x, y, z) in graded-lex
// descending order: the tuples with a larger first exponent come first (a
// tetrahedral number of them), then, within a, those with a larger second
// one (a triangular number), then those with a larger third one
__host__ __device__ constexpr int cidx4(int n, int a, int b, int c)
{
    return (n - a) * (n - a + 1) * (n - a + 2) / 6 + (n - a - b) * (n - a - b + 1) / 2 + (n - a - b - c);
}

// A = C . q^{N-2}: A_ij = sum_{|beta| = N-2} (N-2)!/beta! C_{e_i + e_j + beta} q^beta,
// a symmetric 4 x 4 matrix stored as 00 01 02 03 11 12 13 22 23 33
template <int N>
__device__ __forceinline__ void contract4(const float* c, const float* q, float* A)
{
    constexpr int M = N - 2;
    float pw[4][M + 1];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        pw[i][0] = 1.f;
#pragma unroll
        for (int e = 1; e <= M; e++) pw[i][e] = pw[i][e - 1] * q[i];
    }
#pragma unroll
    for (int i = 0; i < 10; i++) A[i] = 0.f;
#pragma unroll
    for (int b0 = M; b0 >= 0; b0--)
#pragma unroll
        for (int b1 = M - b0; b1 >= 0; b1--)
#pragma unroll
            for (int b2 = M - b0 - b1; b2 >= 0; b2--) {
                const int b3 = M - b0 - b1 - b2;
                const float mb = fact4(M) / (fact4(b0) * fact4(b1) * fact4(b2) * fact4(b3)) * pw[0][b0] * pw[1][b1] *
                                 pw[2][b2] * pw[3][b3];
                int ij = 0;  // the storage order of A
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = i; j < 4; j++, ij++) {
                        const int e0 = b0 + (i == 0) + (j == 0);
                        const int e1 = b1 + (i == 1) + (j == 1);
                        const int e2 = b2 + (i == 2) + (j == 2);
                        A[ij] += mb * c[cidx4(N, e0, e1, e2)];
                    }
            }
}

__device__ __forceinline__ void matvec4(const float* A, const float* v, float* y)
{
    y[0] = A[0] * v[0] + A[1] * v[1] + A[2] * v[2] + A[3] * v[3];
    y[1] = A[1] * v[0] + A[4] * v[1] + A[5] * v[2] + A[6] * v[3];
    y[2] = A[2] * v[0] + A[5] * v[1] + A[7] * v[2] + A[8] * v[3];
    y[3] = A[3] * v[0] + A[6] * v[1] + A[8] * v[2] + A[9] * v[3];
}

__device__ __forceinline__ float dot4(const float* a, const float* b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3];
}

__device__ __forceinline__ void normalise4(float* q)
{
    const float s = rsqrtf(dot4(q, q));
#pragma unroll
    for (int i = 0; i < 4; i++) q[i] *= s;
}

// p = q^T A q with A = C . q^{N-2} (also returned)
template <int N>
__device__ __forceinline__ float form4(const float* c, const float* q, float* A)
{
    contract4<N>(c, q, A);
    float y[4];
    matvec4(A, q, y);
    return dot4(q, y);
}

// tangent basis at unit q: q (x) i, q (x) j, q (x) k
__device__ __forceinline__ void tangent4(const float* q, float (*b)[4])
{
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    b[0][0] = -x; b[0][1] = w;  b[0][2] = z;  b[0][3] = -y;
    b[1][0] = -y; b[1][1] = -z; b[1][2] = w;  b[1][3] = x;
    b[2][0] = -z; b[2][1] = y;  b[2][2] = -x; b[2][3] = w;
}

// smallest eigenvalue of the symmetric 3 x 3 matrix (h00 h01 h02; . h11
// h12; . . h22) by the trigonometric form of the characteristic roots
__device__ __forceinline__ float lmin3(float h00, float h01, float h02, float h11, float h12, float h22)
{
    const float m = (h00 + h11 + h22) * (1.f / 3.f);
    const float a = h00 - m, b = h11 - m, c = h22 - m;
    const float off = h01 * h01 + h02 * h02 + h12 * h12;
    const float pp = (a * a + b * b + c * c + 2.f * off) * (1.f / 6.f);
    if (pp <= 0.f) return m;
    const float s = sqrtf(pp);
    const float is = __fdividef(1.f, s);
    const float B00 = a * is, B11 = b * is, B22 = c * is, B01 = h01 * is, B02 = h02 * is, B12 = h12 * is;
    const float det = B00 * (B11 * B22 - B12 * B12) - B01 * (B01 * B22 - B12 * B02) + B02 * (B01 * B12 - B11 * B02);
    const float r = fminf(1.f, fmaxf(-1.f, 0.5f * det));
    const float phi = acosf(r) * (1.f / 3.f);
    return m + 2.f * s * cosf(phi + 2.0943951f);  // + 2 pi / 3: the smallest root
}

// Newton direction: solves H x = g (H = minus the Riemannian Hessian in the
// basis, symmetric 3 x 3) by LDL^T, first shifting H to 0.05 ||C||_F where
// it is not positive definite; the step is limited to 0.2 rad (a 0.5 rad
// limit overshot more often, and the backtracking costs the whole warp).
__device__ __forceinline__ void newton_dir4(float h00, float h01, float h02, float h11, float h12, float h22,
                                            const float* g, float frob, float* x)
{
    // pivots d_i and their fast reciprocals r_i (the step is only a
    // proposal: backtracking and the monotone fallback guard it)
    const float eps = 1e-6f * frob;
    float d0 = h00, r0 = 0.f, l10 = 0.f, l20 = 0.f, d1 = 0.f, r1 = 0.f, l21 = 0.f, d2 = 0.f;
    bool pd = d0 > eps;
    if (pd) {
        r0 = __fdividef(1.f, d0);
        l10 = h01 * r0; l20 = h02 * r0;
        d1 = h11 - l10 * h01;
        pd = d1 > eps;
        if (pd) {
            r1 = __fdividef(1.f, d1);
            l21 = (h12 - l20 * h01) * r1;
            d2 = h22 - l20 * l20 * d0 - l21 * l21 * d1;
            pd = d2 > eps;
        }
    }
    if (!pd) {
        const float sh = 0.05f * frob - lmin3(h00, h01, h02, h11, h12, h22);
        h00 += sh; h11 += sh; h22 += sh;
        d0 = h00;
        r0 = __fdividef(1.f, d0);
        l10 = h01 * r0; l20 = h02 * r0;
        d1 = h11 - l10 * h01;
        r1 = __fdividef(1.f, d1);
        l21 = (h12 - l20 * h01) * r1;
        d2 = h22 - l20 * l20 * d0 - l21 * l21 * d1;
    }
    const float y0 = g[0], y1 = g[1] - l10 * y0, y2 = g[2] - l20 * y0 - l21 * y1;
    x[2] = __fdividef(y2, d2);
    x[1] = y1 * r1 - l21 * x[2];
    x[0] = y0 * r0 - l10 * x[1] - l20 * x[2];
    const float xn2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    if (xn2 > 0.04f) {
        const float sc = 0.2f * rsqrtf(xn2);
        x[0] *= sc; x[1] *= sc; x[2] *= sc;
    }
}

// gradient (in the basis) and minus the Riemannian Hessian at q; returns
// |gradient|^2
template <int N>
__device__ __forceinline__ float derivs4(const float* A, const float* q, float p, float (*b)[4], float* g, float* h)
{
    float y[4];
    matvec4(A, q, y);
    tangent4(q, b);
    float z[3][4];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        g[a] = N * dot4(b[a], y);
        matvec4(A, b[a], z[a]);
    }
    const float hN = (float)(N * (N - 1));
    h[0] = N * p - hN * dot4(b[0], z[0]);
    h[1] = -hN * dot4(b[0], z[1]);
    h[2] = -hN * dot4(b[0], z[2]);
    h[3] = N * p - hN * dot4(b[1], z[1]);
    h[4] = -hN * dot4(b[1], z[2]);
    h[5] = N * p - hN * dot4(b[2], z[2]);
    return g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
}

// One Riemannian Newton step of q towards a local maximum of p (up to
// max_bt halvings of the step, then a shifted power step); p and A hold the
// value and contraction at q on entry and on return. Returns true, without
// moving, when the tangent gradient is already below 1e-6 ||C||_F.
template <int N>
__device__ __forceinline__ bool newton_step4(const float* c, float frob, float* q, float& p, float* A, int max_bt)
{
    const float tol_p = 1e-7f * frob;
    float b[3][4], g[3], h[6], x[3];
    if (derivs4<N>(A, q, p, b, g, h) <= 1e-12f * frob * frob) return true;
    newton_dir4(h[0], h[1], h[2], h[3], h[4], h[5], g, frob, x);
    float d[4];
#pragma unroll
    for (int i = 0; i < 4; i++) d[i] = x[0] * b[0][i] + x[1] * b[1][i] + x[2] * b[2][i];
    float t = 1.f;
#pragma unroll 1
    for (int bt = 0; bt < max_bt; bt++, t *= 0.5f) {
        float qn[4], An[10];
#pragma unroll
        for (int i = 0; i < 4; i++) qn[i] = q[i] + t * d[i];
        normalise4(qn);
        const float pn = form4<N>(c, qn, An);
        if (pn >= p - tol_p) {
#pragma unroll
            for (int i = 0; i < 4; i++) q[i] = qn[i];
#pragma unroll
            for (int i = 0; i < 10; i++) A[i] = An[i];
            p = pn;
            return false;
        }
    }
    // shifted power step: q <- normalise(A q + (N-1) ||C||_F q)
    float y[4];
    matvec4(A, q, y);
    const float shift = (N - 1) * frob;
#pragma unroll
    for (int i = 0; i < 4; i++) q[i] = y[i] + shift * q[i];
    normalise4(q);
    p = form4<N>(c, q, A);
    return false;
}

// a probe value with the member index m (0..7) in its low 3 mantissa bits:
// a change of at most 7 ulp, far below the FP16 rounding of the keys, that
// lets a running maximum carry the index of the value it holds
__device__ __forceinline__ float tag4(float v, uint32_t m) { return __uint_as_float((__float_as_uint(v) & ~7u) | m); }

// order-preserving 16-bit image of the FP16 rounding of v (larger value,
// larger key), with the low 3 bits replaced by m; and the value back
__device__ __forceinline__ uint32_t hkey(float v, uint32_t m)
{
    const uint32_t h = __half_as_ushort(__float2half_rn(v));
    return ((h ^ ((h & 0x8000u) ? 0xFFFFu : 0x8000u)) & 0xFFF8u) | m;
}
__device__ __forceinline__ float hkey_value(uint32_t k)
{
    const uint32_t h = (k & 0x8000u) ? (k ^ 0x8000u) : (~k & 0xFFFFu);
    return __half2float(__ushort_as_half((unsigned short)h));
}

// table row of member m (0..7) of cell c: the cell of lane quad-position
// t = c & 3 in the tile group G = c >> 2 holds columns 2t, 2t+1 of tiles
// 4G .. 4G+3
__host__ __device__ constexpr int p4_row(int c, int m)
{
    return ((c >> 2) * 4 + (m >> 1)) * 8 + 2 * (c & 3) + (m & 1);
}

struct Probe4Tables {
    const float4* dir;    // [kP4] (w, x, y, z), rows as p4_row
    const __half* phi2h;  // [kP4][p4_kxs(2)] FP16 weighted monomials
    const __half* phi4h;  // [kP4][p4_kxs(4)]
    const __half* phi6h;  // [kP4][p4_kxs(6)]
};

// Top eigenpair of the symmetric 4 x 4 matrix A (00 01 02 03 11 12 13 22
// 23 33) by cyclic Jacobi rotations (each zeroes one off-diagonal entry;
// 6 sweeps leave the off-diagonal part at FP32 rounding). Returns the
// largest eigenvalue and its unit eigenvector in q.
__device__ __forceinline__ float top_eig4(const float* A, float* q)
{
    float a[4][4], v[4][4];
    {
        int ij = 0;
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = i; j < 4; j++, ij++) { a[i][j] = A[ij]; a[j][i] = A[ij]; }
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) v[i][j] = i == j ? 1.f : 0.f;
#pragma unroll 1
    for (int sweep = 0; sweep < 6; sweep++) {
#pragma unroll
        for (int p = 0; p < 3; p++)
#pragma unroll
            for (int r = p + 1; r < 4; r++) {
                const float apr = a[p][r];
                if (apr == 0.f) continue;
                // rotation angle: tan(2 theta) = 2 a_pr / (a_rr - a_pp)
                const float th = (a[r][r] - a[p][p]) / (2.f * apr);
                const float t = (th >= 0.f ? 1.f : -1.f) / (fabsf(th) + sqrtf(th * th + 1.f));
                const float c = rsqrtf(t * t + 1.f), sn = t * c;
#pragma unroll
                for (int k = 0; k < 4; k++) {  // columns p, r
                    const float akp = a[k][p], akr = a[k][r];
                    a[k][p] = c * akp - sn * akr;
                    a[k][r] = sn * akp + c * akr;
                }
#pragma unroll
                for (int k = 0; k < 4; k++) {  // rows p, r
                    const float apk = a[p][k], ark = a[r][k];
                    a[p][k] = c * apk - sn * ark;
                    a[r][k] = sn * apk + c * ark;
                }
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const float vkp = v[k][p], vkr = v[k][r];
                    v[k][p] = c * vkp - sn * vkr;
                    v[k][r] = sn * vkp + c * vkr;
                }
            }
    }
    int b = 0;
#pragma unroll
    for (int i = 1; i < 4; i++)
        if (a[i][i] > a[b][b]) b = i;
    float lam = a[0][0];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        if (i == b) lam = a[i][i];
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (i == b) q[k] = v[k][i];
    }
    normalise4(q);
    return lam;
}

// shared memory: one region of 32-bit words [row][kXStride], column =
// thread, that holds first the staged FP16 input ([KX / 2] rows of half
// pairs) and then the 16-bit cell keys (cells 2r and 2r + 1 in the two
// halves of row r), so that every warp only touches its own columns; then
// the probe directions and the FP16 monomial table. The padding keeps the
// fragment loads and the key stores of a warp in distinct banks.
constexpr int kXStride = kP4Threads + 8;  // 32-bit words
__host__ __device__ constexpr size_t p4_key_bytes(int n)
{
    return sizeof(uint32_t) * (size_t)(kP4Cells / 2 > p4_kx(n) / 2 ? kP4Cells / 2 : p4_kx(n) / 2) * kXStride;
}
// the 16-bit key of cell c of the voxel in column col
__device__ __forceinline__ int key_at(int c, int col) { return 2 * ((c >> 1) * kXStride + col) + (c & 1); }
template <int N>
__host__ __device__ constexpr size_t p4_smem_bytes()
{
    return p4_key_bytes(N) + sizeof(float4) * kP4 + sizeof(__half) * (size_t)kP4 * p4_kxs(N) + sizeof(uint2) * kP4;
}

template <int N>
__global__ void __launch_bounds__(kP4Threads, N >= 6 ? 1 : 2)
k_peakmap4(const float* __restrict__ C, int64_t V, float* __restrict__ score, float* __restrict__ orient,
           float* __restrict__ frob, Probe4Tables tabs)
{
    constexpr int K = ncomp4(N);
    constexpr int KP = p4_kp(N);
    constexpr int KX = p4_kx(N);
    constexpr int KXS = p4_kxs(N);
    constexpr int kStarts = nstarts4(N);
    extern __shared__ __align__(16) unsigned char p4_smem[];
    uint16_t* keys = reinterpret_cast<uint16_t*>(p4_smem);
    uint32_t* xs = reinterpret_cast<uint32_t*>(p4_smem);  // staged input (aliases the keys)
    float4* sdir = reinterpret_cast<float4*>(p4_smem + p4_key_bytes(N));
    __half* phih = reinterpret_cast<__half*>(sdir + kP4);
    // FP16 copies of the directions, only for the 25-degree separation tests
    uint2* sdirh = reinterpret_cast<uint2*>(phih + kP4 * KXS);
    {
        const uint4* src = reinterpret_cast<const uint4*>(N == 2 ? tabs.phi2h : (N == 4 ? tabs.phi4h : tabs.phi6h));
        uint4* dst = reinterpret_cast<uint4*>(phih);
        for (int i = threadIdx.x; i < kP4 * KXS / 8; i += blockDim.x) dst[i] = src[i];
        for (int i = threadIdx.x; i < kP4; i += blockDim.x) {
            const float4 d = tabs.dir[i];
            sdir[i] = d;
            const __half2 a = __floats2half2_rn(d.x, d.y), b = __floats2half2_rn(d.z, d.w);
            sdirh[i] = make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v - threadIdx.x < V;
         v += (int64_t)gridDim.x * blockDim.x) {
        const bool ok = v < V;
        float c[KP];
        float F2 = 0.f;
        {
            int k = 0;
#pragma unroll
            for (int a = N; a >= 0; a--)
#pragma unroll
                for (int b = N - a; b >= 0; b--)
#pragma unroll
                    for (int cc = N - a - b; cc >= 0; cc--) {
                        const int d = N - a - b - cc;
                        const float mult = fact4(N) / (fact4(a) * fact4(b) * fact4(cc) * fact4(d));
                        c[k] = ok ? __ldg(C + (int64_t)k * V + v) : 0.f;
                        F2 += mult * c[k] * c[k];
                        k++;
                    }
#pragma unroll
            for (int k2 = K; k2 < KP; k2++) c[k2] = 0.f;
        }
        const float F = sqrtf(F2);
        float bp = 0.f, bq[4] = {1.f, 0.f, 0.f, 0.f};
        if constexpr (N == 2) {
            if (F > 0.f) {
                float A[10];
#pragma unroll
                for (int i = 0; i < 10; i++) A[i] = c[i];  // C . q^0: the matrix itself
                top_eig4(A, bq);
                bp = form4<N>(c, bq, A);
#pragma unroll 1
                for (int it = 0; it < kP4Polish; it++)
                    if (newton_step4<N>(c, F, bq, bp, A, 4)) break;
            }
        } else {
        // Probe product on the tensor cores: x = C / ||C||_F is staged in
        // FP16 in this thread's column of the key region (rows = component
        // pairs) and loaded as the A fragments of both 16-voxel tiles of the
        // warp; every 8-probe B tile then feeds both. Lane (g, t) holds
        // columns 2t, 2t+1 of each tile for voxel rows g and g+8, so over
        // four tiles it sees exactly the 8 probes of cell 4G + t and keeps
        // their best (value, place) without shuffles.
        {
            const float invF = F > 0.f ? 1.f / F : 0.f;
#pragma unroll
            for (int k = 0; k < KX; k += 2) {
                const __half2 h2 = __floats2half2_rn(k < K ? c[k] * invF : 0.f, k + 1 < K ? c[k + 1] * invF : 0.f);
                xs[(k / 2) * kXStride + threadIdx.x] = *reinterpret_cast<const uint32_t*>(&h2);
            }
            __syncwarp();
            const int g = lane >> 2, t = lane & 3;
            uint32_t a[2][KX / 16][4];
#pragma unroll
            for (int mt = 0; mt < 2; mt++)
#pragma unroll
                for (int ks = 0; ks < KX / 16; ks++) {
                    const uint32_t* r = xs + (8 * ks + t) * kXStride + warp * 32 + 16 * mt + g;
                    a[mt][ks][0] = r[0];
                    a[mt][ks][1] = r[8];
                    a[mt][ks][2] = r[4 * kXStride];
                    a[mt][ks][3] = r[4 * kXStride + 8];
                }
            __syncwarp();
#pragma unroll 1
            for (int G = 0; G < kP4Cells / 4; G++) {
                // running cell bests, each with its member index in the low 3
                // mantissa bits (tag4), so one max carries both
                float mv[2][2];
#pragma unroll
                for (int mt = 0; mt < 2; mt++) mv[mt][0] = mv[mt][1] = -INFINITY;
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const __half* br = phih + ((4 * G + i) * 8 + g) * KXS + 2 * t;
                    uint32_t b0[KX / 16], b1[KX / 16];
#pragma unroll
                    for (int ks = 0; ks < KX / 16; ks++) {
                        b0[ks] = *reinterpret_cast<const uint32_t*>(br + 16 * ks);
                        b1[ks] = *reinterpret_cast<const uint32_t*>(br + 16 * ks + 8);
                    }
#pragma unroll
                    for (int mt = 0; mt < 2; mt++) {
                        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                        for (int ks = 0; ks < KX / 16; ks++) mma_f16(acc, a[mt][ks], b0[ks], b1[ks]);
                        // members 2i, 2i+1 of the cell
                        mv[mt][0] = fmaxf(mv[mt][0], fmaxf(tag4(acc[0], 2 * i), tag4(acc[1], 2 * i + 1)));
                        mv[mt][1] = fmaxf(mv[mt][1], fmaxf(tag4(acc[2], 2 * i), tag4(acc[3], 2 * i + 1)));
                    }
                }
                const int cell = 4 * G + t, col = warp * 32 + g;
#pragma unroll
                for (int mt = 0; mt < 2; mt++) {
                    keys[key_at(cell, col + 16 * mt)] = (uint16_t)hkey(mv[mt][0], __float_as_uint(mv[mt][0]) & 7u);
                    keys[key_at(cell, col + 16 * mt + 8)] = (uint16_t)hkey(mv[mt][1], __float_as_uint(mv[mt][1]) & 7u);
                }
            }
            __syncwarp();
        }
        // starts: the best probe, then by angular suppression over the cell
        // bests: the first pass keeps the cells within 0.2 ||C||_F of the
        // best (an integer compare of keys) that lie farther than 25 degrees
        // from it; each later start is the best kept cell, and the next pass
        // (over the kept cells only) drops those within 25 degrees of it.
        // Start rows are packed 9 bits each.
        uint64_t rows = 0;
        int ns = 1;
        {
            uint32_t best = 0u;
            int bc = 0;
#pragma unroll 8
            for (int cl = 0; cl < kP4Cells; cl++) {
                const uint32_t kk = keys[key_at(cl, threadIdx.x)];
                if (kk > best) { best = kk; bc = cl; }
            }
            int last = p4_row(bc, best & 7u);
            rows = (uint64_t)last;
            const uint32_t thr = hkey(hkey_value(best) - p4_margin(N), 0u);
            uint64_t alive = 0ull;
            uint32_t bk = 0u;
            int bcell = -1;
            {
                const float4 ds = sdir[last];
#pragma unroll 4
                for (int cl = 0; cl < kP4Cells; cl++) {
                    const uint32_t kk = keys[key_at(cl, threadIdx.x)];
                    if (kk < thr) continue;
                    const uint2 dh = sdirh[p4_row(cl, kk & 7u)];
                    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&dh.x));
                    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&dh.y));
                    const float dt = fabsf(a.x * ds.x + a.y * ds.y + b.x * ds.z + b.y * ds.w);
                    if (dt < kP4SepCos) {
                        alive |= 1ull << cl;
                        if (kk > bk) { bk = kk; bcell = cl; }
                    }
                }
            }
#pragma unroll 1
            for (int s = 1; s < kStarts && bcell >= 0; s++) {
                last = p4_row(bcell, bk & 7u);
                rows |= (uint64_t)last << (9 * s);
                ns = s + 1;
                alive &= ~(1ull << bcell);
                if (s + 1 == kStarts) break;
                const float4 ds = sdir[last];
                bk = 0u;
                bcell = -1;
                for (uint64_t m = alive; m; m &= m - 1) {
                    const int cl = __ffsll((long long)m) - 1;
                    const uint32_t kk = keys[key_at(cl, threadIdx.x)];
                    const uint2 dh = sdirh[p4_row(cl, kk & 7u)];
                    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&dh.x));
                    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&dh.y));
                    const float dt = fabsf(a.x * ds.x + a.y * ds.y + b.x * ds.z + b.y * ds.w);
                    if (dt >= kP4SepCos) alive &= ~(1ull << cl);
                    else if (kk > bk) { bk = kk; bcell = cl; }
                }
            }
        }
        __syncwarp();  // the key rows are restaged by the next voxel block
        if (F > 0.f) {
            float bA[10];
            bp = -INFINITY;
#pragma unroll 1
            for (int s = 0; s < ns; s++) {
                const float4 d4 = sdir[(int)((rows >> (9 * s)) & 511u)];
                float q[4] = {d4.x, d4.y, d4.z, d4.w}, A[10];
                float p = form4<N>(c, q, A);
#pragma unroll 1
                for (int it = 0; it < kP4Pre; it++)
                    if (newton_step4<N>(c, F, q, p, A, 2)) break;
                if (p > bp) {
                    bp = p;
#pragma unroll
                    for (int i = 0; i < 4; i++) bq[i] = q[i];
#pragma unroll
                    for (int i = 0; i < 10; i++) bA[i] = A[i];
                }
            }
#pragma unroll 1
            for (int it = 0; it < kP4Polish; it++)
                if (newton_step4<N>(c, F, bq, bp, bA, 4)) break;
        }
        }  // N > 2
        // canonical sign: the first non-zero of (w, x, y, z) positive
        const bool neg = bq[0] < 0.f ||
                         (bq[0] == 0.f && (bq[1] < 0.f || (bq[1] == 0.f && (bq[2] < 0.f || (bq[2] == 0.f && bq[3] < 0.f)))));
        if (neg) {
#pragma unroll
            for (int i = 0; i < 4; i++) bq[i] = -bq[i];
        }
        if (ok) {
            score[v] = bp;
#pragma unroll
            for (int i = 0; i < 4; i++) orient[(int64_t)i * V + v] = bq[i];
            if (frob) frob[v] = F;
        }
    }
}

// ---------------------------------------------------------------- host --

// 512 super-Fibonacci quaternions (the sampling of the rotation quadrature,
// without the cube group) with w >= 0, grouped into 64 cells of 8: each
// cell is the lowest-index unassigned probe and its 7 nearest unassigned
// neighbours (distance |q . q'|, as q ~ -q), member m of cell c placed at
// table row p4_row(c, m). Layout: directions [kP4] float4, then the FP32
// weighted monomials mult(alpha) q^alpha for n = 2, 4 and 6, [kP4][p4_kp(n)].
static void build_probe4(std::vector<float>& out, size_t off[4])
{
    std::vector<double> q;
    rotation_set(kP4, false, q);
    for (int i = 0; i < kP4; i++)
        if (q[4 * i] < 0)
            for (int k = 0; k < 4; k++) q[4 * i + k] = -q[4 * i + k];
    std::vector<int> order;
    std::vector<char> used(kP4, 0);
    for (int seed = 0; seed < kP4; seed++) {
        if (used[seed]) continue;
        std::vector<std::pair<double, int>> cand;
        for (int j = 0; j < kP4; j++)
            if (!used[j]) {
                double d = 0;
                for (int k = 0; k < 4; k++) d += q[4 * seed + k] * q[4 * j + k];
                cand.push_back({-std::fabs(d), j});
            }
        std::sort(cand.begin(), cand.end());
        for (int m = 0; m < 8 && m < (int)cand.size(); m++) {
            order.push_back(cand[m].second);
            used[cand[m].second] = 1;
        }
    }
    // member m of cluster c goes to table row p4_row(c, m)
    std::vector<int> src(kP4);
    for (int c = 0; c < kP4Cells; c++)
        for (int m = 0; m < 8; m++) src[p4_row(c, m)] = order[8 * c + m];
    out.clear();
    off[0] = 0;
    for (int j : src)
        for (int k = 0; k < 4; k++) out.push_back((float)q[4 * j + k]);
    int slot = 1;
    for (int n : {2, 4, 6}) {
        off[slot++] = out.size();
        std::vector<int> e;
        exponents4(n, e);
        const int K = (int)e.size() / 4;
        for (int j : src) {
            for (int k = 0; k < K; k++) {
                double mult = std::tgamma(n + 1.0), mono = 1.0;
                for (int d = 0; d < 4; d++) {
                    mult /= std::tgamma(e[4 * k + d] + 1.0);
                    mono *= std::pow(q[4 * j + d], e[4 * k + d]);
                }
                out.push_back((float)(mult * mono));
            }
            for (int k = K; k < p4_kp(n); k++) out.push_back(0.f);
        }
    }
}

__global__ void k_phi4_half(const float* __restrict__ phi, int KP, int K, int KXS, __half* __restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kP4 * KXS; i += gridDim.x * blockDim.x) {
        const int j = i / KXS, k = i - j * KXS;
        out[i] = __float2half_rn(k < K ? phi[j * KP + k] : 0.f);
    }
}

void upload_probe_tables4(ttm_ctx* ctx)
{
    std::vector<float> h;
    size_t off[4];
    build_probe4(h, off);
    DevBuf f32;
    f32.alloc(h.size() * sizeof(float));
    TTM_CUDA_TRY(cudaMemcpy(f32.p, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
    const size_t dir_bytes = sizeof(float4) * kP4;
    const size_t h2 = sizeof(__half) * (size_t)kP4 * p4_kxs(2), h4 = sizeof(__half) * (size_t)kP4 * p4_kxs(4);
    const size_t h6 = sizeof(__half) * (size_t)kP4 * p4_kxs(6);
    ctx->probe4.alloc(dir_bytes + h2 + h4 + h6);
    TTM_CUDA_TRY(cudaMemcpy(ctx->probe4.p, f32.p, dir_bytes, cudaMemcpyDeviceToDevice));
    unsigned char* base = ctx->probe4.as<unsigned char>();
    k_phi4_half<<<64, 256>>>(f32.as<float>() + off[1], p4_kp(2), ncomp4(2), p4_kxs(2),
                             reinterpret_cast<__half*>(base + dir_bytes));
    TTM_LAUNCH_CHECK();
    k_phi4_half<<<64, 256>>>(f32.as<float>() + off[2], p4_kp(4), ncomp4(4), p4_kxs(4),
                             reinterpret_cast<__half*>(base + dir_bytes + h2));
    TTM_LAUNCH_CHECK();
    k_phi4_half<<<64, 256>>>(f32.as<float>() + off[3], p4_kp(6), ncomp4(6), p4_kxs(6),
                             reinterpret_cast<__half*>(base + dir_bytes + h2 + h4));
    TTM_LAUNCH_CHECK();
    TTM_CUDA_TRY(cudaDeviceSynchronize());
    ctx->probe4_off[0] = 0;
    ctx->probe4_off[1] = dir_bytes;
    ctx->probe4_off[2] = dir_bytes + h2;
    ctx->probe4_off[3] = dir_bytes + h2 + h4;
}

void peakmap4_run(ttm_ctx* ctx, int n, const float* C, int64_t V, float* score, float* orient, float* frob,
                  cudaStream_t st)
{
    const unsigned char* base = ctx->probe4.as<unsigned char>();
    const Probe4Tables t{reinterpret_cast<const float4*>(base + ctx->probe4_off[0]),
                         reinterpret_cast<const __half*>(base + ctx->probe4_off[1]),
                         reinterpret_cast<const __half*>(base + ctx->probe4_off[2]),
                         reinterpret_cast<const __half*>(base + ctx->probe4_off[3])};
    const int64_t blocks = std::max<int64_t>(1, ceil_div(V, kP4Threads));
    // two resident CTAs per SM (one at n = 6); a grid stride balances the
    // uneven Newton work
    const int64_t grid = std::min<int64_t>(blocks, (int64_t)ctx->num_sms * 16);
#define TTM_P4_LAUNCH(N_)                                                                                       \
    {                                                                                                            \
        const size_t smem = p4_smem_bytes<N_>();                                                                 \
        TTM_CUDA_TRY(cudaFuncSetAttribute(k_peakmap4<N_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        k_peakmap4<N_><<<(unsigned)grid, kP4Threads, smem, st>>>(C, V, score, orient, frob, t);                 \
    }
    switch (n) {
        case 2: TTM_P4_LAUNCH(2); break;
        case 4: TTM_P4_LAUNCH(4); break;
        case 6: TTM_P4_LAUNCH(6); break;
        default: throw Error{E_UNSUPPORTED, "the quaternion maximiser is built for n = 2, 4 and 6"};
    }
#undef TTM_P4_LAUNCH
    TTM_LAUNCH_CHECK();
}

}  // namespace ttm
