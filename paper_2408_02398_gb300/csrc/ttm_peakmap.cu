// ttm_peakmap.cu -- per-voxel contraction and maximisation over unit
// directions (Sec. 3.1 and 3.2):
//   F(x) = ||C(x)||_F,  s(x) = max_{|u|=1} p_x(u),  u*(x) = argmax,
//   p_x(u) = C(x) . u^{(x)n} = sum_alpha mult(alpha) C_alpha(x) u^alpha.
//
// One thread per voxel, components loaded structure-of-arrays (coalesced),
// persistent CTAs. The form is evaluated at P = 128 fixed probe directions on
// the half-sphere (p is even) as a tensor-core product per warp. The probes
// form 16 cells of 8 neighbours, laid out so that one lane holds a whole
// cell; only each cell's best probe is kept (a 16-bit key in shared
// memory). The starts are the best probe and, by angular suppression, up to
// NS - 1 more (NS = 2 for n = 2, 3 otherwise): the best cell best farther
// than 20 degrees from the starts already taken, if within 0.2 ||C||_F of
// the best. The starts get up to two Newton steps each, in turn (one
// inlined copy of the step), and the best is polished to convergence. The
// derivatives come from the contraction A = C . u^{n-2} (a symmetric 3x3
// matrix): p = u^T A u, grad p = n A u, Hess p = n (n-1) A. Each polish step
// is a Riemannian Newton step in a branchless orthonormal tangent basis,
// limited to 0.2 rad; where the tangent Hessian is not negative definite it is shifted
// until it is (a Levenberg-Marquardt direction) and the step is taken at the
// full 0.2 rad, the step is halved until p does not decrease, and a shifted
// power step (SS-HOPM, shift (n-1)||C||_F, never decreasing) is the last
// resort.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_fp16.h>

#include "mlp_mma.cuh"
#include "ttm_internal.h"

namespace ttm {

constexpr int kProbes = 128;
constexpr int kPmThreads = 128;
constexpr int kPreIters = 2;      // cheap polish of every start
constexpr int kNewtonIters = 10;  // full polish of the best one
// probes more than this fraction of ||C||_F below the best probe are not
// considered as starts
constexpr float kStartMargin = 0.2f;
// extra starts lie farther than this from the starts already chosen
constexpr double kStartSepDeg = 20.0;
constexpr float kStartSepCos = 0.93969262f;  // cos(20 degrees)

__host__ __device__ constexpr int ncomp3(int n) { return (n + 1) * (n + 2) / 2; }
// starts polished per voxel: order 2 has a single maximum pair; higher
// orders have more, narrower maxima (and the FP16 probe values can reorder
// near-equal candidates)
__host__ __device__ constexpr int nstarts(int n) { return n >= 4 ? 3 : 2; }
__host__ __device__ constexpr int kpad(int n) { return (ncomp3(n) + 3) / 4 * 4; }
__host__ __device__ constexpr float factf(int n) { return n <= 1 ? 1.f : n * factf(n - 1); }
// position of exponents (a, b, n-a-b) in graded-lex descending order
__host__ __device__ constexpr int cidx(int n, int a, int b) { return (n - a) * (n - a + 1) / 2 + (n - a - b); }

// probe cells: the 8 probes of cell c are the columns 2t, 2t+1 (t = c & 3)
// of the 8-probe tensor-core tiles 4G .. 4G+3 (G = c >> 2), i.e. exactly
// the columns one lane of a warp holds in those tiles
constexpr int kCells = 128 / 8;
__host__ __device__ constexpr int cell_row(int c, int m) { return ((c >> 2) * 4 + (m >> 1)) * 8 + 2 * (c & 3) + (m & 1); }

// A = C . u^{N-2}: A_ij = sum_beta (N-2)!/beta! C_{e_i + e_j + beta} u^beta,
// stored xx, xy, xz, yy, yz, zz
template <int N>
__device__ __forceinline__ void contract2(const float* c, float ux, float uy, float uz, float* A)
{
    constexpr int M = N - 2;
    float px[M + 1], py[M + 1], pz[M + 1];
    px[0] = py[0] = pz[0] = 1.f;
#pragma unroll
    for (int e = 1; e <= M; e++) { px[e] = px[e - 1] * ux; py[e] = py[e - 1] * uy; pz[e] = pz[e - 1] * uz; }
#pragma unroll
    for (int i = 0; i < 6; i++) A[i] = 0.f;
#pragma unroll
    for (int a = M; a >= 0; a--) {
#pragma unroll
        for (int b = M - a; b >= 0; b--) {
            const int cc = M - a - b;
            const float mb = factf(M) / (factf(a) * factf(b) * factf(cc)) * px[a] * py[b] * pz[cc];
            A[0] += mb * c[cidx(N, a + 2, b)];
            A[1] += mb * c[cidx(N, a + 1, b + 1)];
            A[2] += mb * c[cidx(N, a + 1, b)];
            A[3] += mb * c[cidx(N, a, b + 2)];
            A[4] += mb * c[cidx(N, a, b + 1)];
            A[5] += mb * c[cidx(N, a, b)];
        }
    }
}

// p = u^T A u at u, with A = C . u^{N-2} (also returned)
template <int N>
__device__ __forceinline__ float form_at(const float* c, float ux, float uy, float uz, float* A)
{
    contract2<N>(c, ux, uy, uz, A);
    return ux * (A[0] * ux + A[1] * uy + A[2] * uz) + uy * (A[1] * ux + A[3] * uy + A[4] * uz) +
           uz * (A[2] * ux + A[4] * uy + A[5] * uz);
}

__device__ __forceinline__ void normalise3(float& x, float& y, float& z)
{
    float s = rsqrtf(x * x + y * y + z * z);
    x *= s; y *= s; z *= s;
}

// up to iters polish steps of u towards a local maximum of p; p and A hold
// the value and contraction at u on entry and on return. Returns whether
// the tangent gradient fell below its tolerance.
template <int N>
__device__ __forceinline__ bool polish(const float* c, float frob, float& ux, float& uy, float& uz, float& p,
                                       float* A, int iters)
{
    // |tangent gradient| <= 3e-6 ||C||_F: the direction is then within
    // 3e-6 / curvature rad of the maximum (0.17 degrees where the curvature is
    // 1e-3 ||C||_F, the flattest maximum whose orientation is defined)
    const float tol_g2 = 9e-12f * frob * frob;
    const float tol_p = 1e-7f * frob;
    const float hN = (float)(N * (N - 1));
#pragma unroll 1
    for (int it = 0; it < iters; it++) {
        const float ax = A[0] * ux + A[1] * uy + A[2] * uz;
        const float ay = A[1] * ux + A[3] * uy + A[4] * uz;
        const float az = A[2] * ux + A[4] * uy + A[5] * uz;
        // grad = N A u, Hess = N (N-1) A, u . grad = N p.
        // Tangent basis without branches (Duff et al. 2017, "Building an
        // orthonormal basis, revisited"): with s = sign(u_z), a = -1/(s + u_z)
        // and b = u_x u_y a, the vectors (1 + s u_x^2 a, s b, -s u_x) and
        // (b, s + u_y^2 a, -u_y) are orthonormal and orthogonal to the unit u;
        // |s + u_z| >= 1, so nothing cancels, at the poles included.
        const float sg = copysignf(1.f, uz);
        const float ra = __fdividef(-1.f, sg + uz);
        const float rb = ux * uy * ra;
        const float b0x = fmaf(sg * ux, ux * ra, 1.f);
        const float b0y = sg * rb;
        const float b0z = -sg * ux;
        const float b1x = rb;
        const float b1y = fmaf(uy * uy, ra, sg);
        const float b1z = -uy;
        const float g0 = N * (b0x * ax + b0y * ay + b0z * az);
        const float g1 = N * (b1x * ax + b1y * ay + b1z * az);
        if (g0 * g0 + g1 * g1 <= tol_g2) return true;
        const float a0x = A[0] * b0x + A[1] * b0y + A[2] * b0z;
        const float a0y = A[1] * b0x + A[3] * b0y + A[4] * b0z;
        const float a0z = A[2] * b0x + A[4] * b0y + A[5] * b0z;
        const float a1x = A[0] * b1x + A[1] * b1y + A[2] * b1z;
        const float a1y = A[1] * b1x + A[3] * b1y + A[4] * b1z;
        const float a1z = A[2] * b1x + A[4] * b1y + A[5] * b1z;
        // minus the Riemannian Hessian in the basis: N p I - N(N-1) B^T A B
        float h00 = N * p - hN * (b0x * a0x + b0y * a0y + b0z * a0z);
        const float h01 = -hN * (b1x * a0x + b1y * a0y + b1z * a0z);
        float h11 = N * p - hN * (b1x * a1x + b1y * a1y + b1z * a1z);
        // pure Newton where it is positive definite, else shift it to 0.05 ||C||_F
        const float mid = 0.5f * (h00 + h11), dif = 0.5f * (h00 - h11);
        const float lmin = mid - sqrtf(dif * dif + h01 * h01);
        const bool shifted = lmin <= 1e-6f * frob;
        if (shifted) { const float sh = 0.05f * frob - lmin; h00 += sh; h11 += sh; }
        const float idet = __frcp_rn(h00 * h11 - h01 * h01);
        float x0 = (h11 * g0 - h01 * g1) * idet;
        float x1 = (h00 * g1 - h01 * g0) * idet;
        const float xn2 = x0 * x0 + x1 * x1;
        // |step| <= 0.2 rad; a shifted (not negative definite) step is taken
        // at that full length: far from a maximum along a flat ridge the
        // shifted step is tiny, and backtracking keeps p from decreasing.
        // (A 0.5 rad cap overshot more often and cost backtracking
        // evaluations, which the whole warp pays for.)
        if (xn2 > 0.04f || (shifted && xn2 > 0.f)) { const float sc = 0.2f * rsqrtf(xn2); x0 *= sc; x1 *= sc; }
        const float dx = x0 * b0x + x1 * b1x, dy = x0 * b0y + x1 * b1y, dz = x0 * b0z + x1 * b1z;
        bool moved = false;
        float t = 1.f;
#pragma unroll 1
        for (int bt = 0; bt < 4 && !moved; bt++, t *= 0.5f) {
            float nx = ux + t * dx, ny = uy + t * dy, nz = uz + t * dz;
            normalise3(nx, ny, nz);
            float An[6];
            const float pn = form_at<N>(c, nx, ny, nz, An);
            if (pn >= p - tol_p) {
                ux = nx; uy = ny; uz = nz; p = pn;
#pragma unroll
                for (int i = 0; i < 6; i++) A[i] = An[i];
                moved = true;
            }
        }
        if (!moved) {
            // shifted power step: u <- normalise(A u + (N-1) ||C||_F u), never decreases p
            const float shift = (N - 1) * frob;
            float nx = ax + shift * ux, ny = ay + shift * uy, nz = az + shift * uz;
            normalise3(nx, ny, nz);
            ux = nx; uy = ny; uz = nz;
            p = form_at<N>(c, ux, uy, uz, A);
        }
    }
    return false;
}

// Largest eigenvalue of the symmetric 3x3 matrix A (xx, xy, xz, yy, yz, zz)
// by the trigonometric form of the characteristic roots, and a unit
// eigenvector: the longest cross product of two rows of A - lambda I (the
// rows span the orthogonal complement of the eigenvector). Where A is a
// multiple of I every direction is an eigenvector and e_z is returned.
__device__ __forceinline__ float top_eig3(const float* A, float& ux, float& uy, float& uz)
{
    const float m = (A[0] + A[3] + A[5]) * (1.f / 3.f);
    const float a = A[0] - m, b = A[3] - m, c = A[5] - m;
    const float off = A[1] * A[1] + A[2] * A[2] + A[4] * A[4];
    const float pp = (a * a + b * b + c * c + 2.f * off) * (1.f / 6.f);
    ux = 0.f; uy = 0.f; uz = 1.f;
    if (!(pp > 0.f)) return m;
    const float sq = sqrtf(pp), is = 1.f / sq;
    const float B00 = a * is, B11 = b * is, B22 = c * is, B01 = A[1] * is, B02 = A[2] * is, B12 = A[4] * is;
    const float det = B00 * (B11 * B22 - B12 * B12) - B01 * (B01 * B22 - B12 * B02) + B02 * (B01 * B12 - B11 * B02);
    const float r = fminf(1.f, fmaxf(-1.f, 0.5f * det));
    const float lam = m + 2.f * sq * cosf(acosf(r) * (1.f / 3.f));
    const float a0 = A[0] - lam, a1 = A[1], a2 = A[2];  // row 0 of A - lambda I
    const float b0 = A[1], b1 = A[3] - lam, b2 = A[4];  // row 1
    const float c0 = A[2], c1 = A[4], c2 = A[5] - lam;  // row 2
    float best = 0.f;
    auto take = [&](float x0, float x1, float x2, float y0, float y1, float y2) {
        const float cx = x1 * y2 - x2 * y1, cy = x2 * y0 - x0 * y2, cz = x0 * y1 - x1 * y0;
        const float n2 = cx * cx + cy * cy + cz * cz;
        if (n2 > best) { best = n2; ux = cx; uy = cy; uz = cz; }
    };
    take(a0, a1, a2, b0, b1, b2);
    take(a0, a1, a2, c0, c1, c2);
    take(b0, b1, b2, c0, c1, c2);
    if (best > 0.f) {
        const float s = rsqrtf(best);
        ux *= s; uy *= s; uz *= s;
    } else {
        ux = 0.f; uy = 0.f; uz = 1.f;
    }
    return lam;
}

// probe tables: directions [kProbes][4] (x, y, z, 0) and weighted monomials
// [kProbes][kpad(n)] for n = 2, 4, 6, in global memory
struct ProbeTables {
    const float4* dir;
    const float* phi2;
    const float* phi4;
    const float* phi6;
    const uint4* far;          // [kProbes] 128-bit rows: probes j with |d_i . d_j| < cos(kStartSepDeg)
    // FP16 copies [kProbes][pm_kxs(n)] (components beyond K and the row
    // padding zero) for the tensor-core probe product
    const __half* phi2h;
    const __half* phi4h;
    const __half* phi6h;
};

// one region of 32-bit words [row][kPvStride], column = thread: first the
// staged FP16 input (pm_kx / 2 rows of component pairs), then the 16-bit
// cell keys (cells 2r and 2r + 1 in the two halves of row r), so that every
// warp only touches its own columns; the padding (136 words per row) keeps
// the fragment loads and the key stores of a warp in distinct banks
constexpr int kPvStride = kPmThreads + 8;
__host__ __device__ constexpr int pm_kx(int n) { return (ncomp3(n) + 15) / 16 * 16; }
__host__ __device__ constexpr int pm_kxs(int n) { return pm_kx(n) + 8; }
__host__ __device__ constexpr int pm_rows(int n) { return pm_kx(n) / 2 > kCells / 2 ? pm_kx(n) / 2 : kCells / 2; }
__host__ __device__ constexpr size_t pm_smem_bytes(int n)
{
    return sizeof(uint32_t) * (size_t)pm_rows(n) * kPvStride + sizeof(__half) * (size_t)kProbes * pm_kxs(n);
}
// a probe value with the member index m (0..7) in its low 3 mantissa bits:
// a change of at most 7 ulp, far below the FP16 rounding of the keys, that
// lets a running maximum carry the index of the value it holds
__device__ __forceinline__ float pm_tag(float v, uint32_t m) { return __uint_as_float((__float_as_uint(v) & ~7u) | m); }
// the 16-bit key of cell c of the voxel in column col
__device__ __forceinline__ int pm_key_at(int c, int col) { return 2 * ((c >> 1) * kPvStride + col) + (c & 1); }
// order-preserving 16-bit image of the FP16 rounding of v with the low 3
// bits replaced by m (a cell member), and the value back
__device__ __forceinline__ uint32_t pm_hkey(float v, uint32_t m)
{
    const uint32_t h = __half_as_ushort(__float2half_rn(v));
    return ((h ^ ((h & 0x8000u) ? 0xFFFFu : 0x8000u)) & 0xFFF8u) | m;
}
__device__ __forceinline__ float pm_hkey_value(uint32_t k)
{
    const uint32_t h = (k & 0x8000u) ? (k ^ 0x8000u) : (~k & 0xFFFFu);
    return __half2float(__ushort_as_half((unsigned short)h));
}

// which voxels a k_peakmap launch visits
enum PmMode { PM_ALL = 0, PM_LIST = 1, PM_SWEEP = 2, PM_BOX = 3 };

// PM_ALL: every voxel. PM_LIST: the first min(*list_count, list_cap)
// entries of list. PM_SWEEP: only if *list_count > list_cap (the list
// overflowed), every voxel whose score holds the NaN placed there by the
// learned maximiser. PM_BOX: the voxels of a box of the C grid (row
// lengths Yin, Xin), written to a grid with rows Yout, Xout and component
// stride Vout (the tomogram grid of a zero-padded working grid).
struct PmGeom {
    int mode = PM_ALL;
    const uint32_t* list = nullptr;
    const unsigned long long* list_count = nullptr;
    int64_t list_cap = 0;
    int z0 = 0, y0 = 0, x0 = 0, bz = 0, by = 0, bx = 0;
    int Yin = 0, Xin = 0, Yout = 0, Xout = 0;
    int64_t Vout = 0;
};

template <int N>
__global__ void __launch_bounds__(kPmThreads, N >= 6 ? 5 : 7)
k_peakmap(const float* __restrict__ C, int64_t V, float* __restrict__ score, float* __restrict__ orient,
          float* __restrict__ frob, ProbeTables tabs, PmGeom geo)
{
    const int mode = geo.mode;
    if (mode == PM_SWEEP && (int64_t)*geo.list_count <= geo.list_cap) return;
    const int64_t n_items = mode == PM_LIST ? min((int64_t)*geo.list_count, geo.list_cap)
                          : mode == PM_BOX ? (int64_t)geo.bz * geo.by * geo.bx : V;
    const int64_t Vo = mode == PM_BOX ? geo.Vout : V;
    constexpr int K = ncomp3(N);
    constexpr int KP = kpad(N);
    constexpr int KX = pm_kx(N);
    constexpr int KXS = pm_kxs(N);
    constexpr int kStarts = nstarts(N);
    __shared__ float4 sdir[kProbes];
    // xs / keys: the staged input, then the cell keys (see pm_key_at);
    // phih: [kProbes][KXS] FP16 weighted monomials
    extern __shared__ __align__(16) __half pm_smem[];
    uint32_t* xs = reinterpret_cast<uint32_t*>(pm_smem);
    uint16_t* keys = reinterpret_cast<uint16_t*>(pm_smem);
    __half* phih = pm_smem + 2 * pm_rows(N) * kPvStride;
    {
        const __half* ph = N == 2 ? tabs.phi2h : (N == 4 ? tabs.phi4h : tabs.phi6h);
        const uint4* src = reinterpret_cast<const uint4*>(ph);
        uint4* dst = reinterpret_cast<uint4*>(phih);
        for (int i = threadIdx.x; i < kProbes * KXS / 8; i += blockDim.x) dst[i] = src[i];
        for (int i = threadIdx.x; i < kProbes; i += blockDim.x) sdir[i] = tabs.dir[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // persistent: each CTA walks voxel blocks with a grid stride
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t - threadIdx.x < n_items;
         t += (int64_t)gridDim.x * blockDim.x) {
        bool ok = t < n_items;
        int64_t v = t, vo = t;
        if (mode == PM_LIST && ok) vo = v = geo.list[t];
        if (mode == PM_SWEEP && ok) ok = isnan(score[v]);
        if (mode == PM_BOX && ok) {
            const int xx = (int)(t % geo.bx);
            const int64_t r = t / geo.bx;
            const int yy = (int)(r % geo.by), zz = (int)(r / geo.by);
            const int z = geo.z0 + zz, y = geo.y0 + yy, x = geo.x0 + xx;
            v = ((int64_t)z * geo.Yin + y) * geo.Xin + x;
            vo = ((int64_t)z * geo.Yout + y) * geo.Xout + x;
        }
        float c[KP];
        float F2 = 0.f;
        {
            int k = 0;
#pragma unroll
            for (int a = N; a >= 0; a--)
#pragma unroll
                for (int b = N - a; b >= 0; b--) {
                    const int cc = N - a - b;
                    const float mult = factf(N) / (factf(a) * factf(b) * factf(cc));
                    c[k] = ok ? __ldg(C + (int64_t)k * V + v) : 0.f;
                    F2 += mult * c[k] * c[k];
                    k++;
                }
#pragma unroll
            for (int k2 = K; k2 < KP; k2++) c[k2] = 0.f;
        }
        const float F = sqrtf(F2);
        float best = 0.f, bx = 0.f, by = 0.f, bz = 1.f;
        if constexpr (N == 2) {
            // n = 2: p(u) = u^T A u with A_ij = C_{e_i + e_j}, whose maximum
            // over unit u is the top eigenpair of A; Newton polishes the
            // closed form to FP32 convergence
            if (F > 0.f) {
                const float A2[6] = {c[0], c[1], c[2], c[3], c[4], c[5]};
                top_eig3(A2, bx, by, bz);
                float A[6];
                best = form_at<N>(c, bx, by, bz, A);
                polish<N>(c, F, bx, by, bz, best, A, kNewtonIters);
            }
        } else {
            // Probe values p_j / ||C||_F of the warp's 32 voxels on the tensor
            // cores: x = C / ||C||_F (|x_k| <= 1) is staged in FP16 in this
            // thread's column (rows = component pairs) and loaded as the A
            // fragments of both 16-voxel tiles; every 8-probe B tile feeds both.
            // Lane (g, t) holds columns 2t, 2t+1 of each tile for voxel rows g
            // and g+8, so over four tiles it sees exactly the 8 probes of cell
            // 4G + t and keeps their best (value, member) without shuffles; the
            // cell bests go to shared memory as 16-bit keys.
            {
                const float invF = F > 0.f ? 1.f / F : 0.f;
    #pragma unroll
                for (int k = 0; k < KX; k += 2) {
                    const __half2 h2 = __floats2half2_rn(k < K ? c[k] * invF : 0.f, k + 1 < K ? c[k + 1] * invF : 0.f);
                    xs[(k / 2) * kPvStride + threadIdx.x] = *reinterpret_cast<const uint32_t*>(&h2);
                }
                __syncwarp();
                const int g = lane >> 2, t = lane & 3;
                uint32_t a[2][KX / 16][4];
    #pragma unroll
                for (int mt = 0; mt < 2; mt++)
    #pragma unroll
                    for (int ks = 0; ks < KX / 16; ks++) {
                        const uint32_t* r = xs + (8 * ks + t) * kPvStride + warp * 32 + 16 * mt + g;
                        a[mt][ks][0] = r[0];
                        a[mt][ks][1] = r[8];
                        a[mt][ks][2] = r[4 * kPvStride];
                        a[mt][ks][3] = r[4 * kPvStride + 8];
                    }
                __syncwarp();
                // unrolled for n <= 4; at n = 6 (5 CTAs per SM) the unrolled
                // loop measured 5 % slower
    #pragma unroll (N >= 6 ? 1 : kCells / 4)
                for (int G = 0; G < kCells / 4; G++) {
                    // running cell bests, each with its member index in the low
                    // 3 mantissa bits (pm_tag), so one max carries both
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
                            mv[mt][0] = fmaxf(mv[mt][0], fmaxf(pm_tag(acc[0], 2 * i), pm_tag(acc[1], 2 * i + 1)));
                            mv[mt][1] = fmaxf(mv[mt][1], fmaxf(pm_tag(acc[2], 2 * i), pm_tag(acc[3], 2 * i + 1)));
                        }
                    }
                    const int cell = 4 * G + t, col = warp * 32 + g;
    #pragma unroll
                    for (int mt = 0; mt < 2; mt++) {
                        keys[pm_key_at(cell, col + 16 * mt)] = (uint16_t)pm_hkey(mv[mt][0], __float_as_uint(mv[mt][0]) & 7u);
                        keys[pm_key_at(cell, col + 16 * mt + 8)] = (uint16_t)pm_hkey(mv[mt][1], __float_as_uint(mv[mt][1]) & 7u);
                    }
                }
                __syncwarp();
            }
            // Starts by angular suppression over the cell bests: the best probe,
            // then the best cell best farther than kStartSepDeg from every start
            // taken and within kStartMargin ||C||_F of the best. The first pass
            // keeps the cells within the margin (an integer compare of keys) and
            // farther than kStartSepDeg from the best; each later pass, over the
            // kept cells only, drops those near the newest start.
            int sj[kStarts];
            bool live[kStarts];
            {
                uint32_t best = 0u;
                int bc = 0;
    #pragma unroll
                for (int cl = 0; cl < kCells; cl++) {
                    const uint32_t kk = keys[pm_key_at(cl, threadIdx.x)];
                    if (kk > best) { best = kk; bc = cl; }
                }
                sj[0] = cell_row(bc, best & 7u);
                live[0] = true;
    #pragma unroll
                for (int s = 1; s < kStarts; s++) { sj[s] = sj[0]; live[s] = false; }
                const uint32_t thr = pm_hkey(pm_hkey_value(best) - kStartMargin, 0u);
                uint32_t alive = 0u, bk = 0u;
                int bcell = -1;
                {
                    const float4 ds = sdir[sj[0]];
    #pragma unroll
                    for (int cl = 0; cl < kCells; cl++) {
                        const uint32_t kk = keys[pm_key_at(cl, threadIdx.x)];
                        if (kk < thr) continue;
                        const float4 dj = sdir[cell_row(cl, kk & 7u)];
                        if (fabsf(dj.x * ds.x + dj.y * ds.y + dj.z * ds.z) < kStartSepCos) {
                            alive |= 1u << cl;
                            if (kk > bk) { bk = kk; bcell = cl; }
                        }
                    }
                }
    #pragma unroll
                for (int s = 1; s < kStarts; s++) {
                    if (bcell < 0) break;
                    sj[s] = cell_row(bcell, bk & 7u);
                    live[s] = true;
                    alive &= ~(1u << bcell);
                    if (s + 1 == kStarts) break;
                    const float4 ds = sdir[sj[s]];
                    bk = 0u;
                    bcell = -1;
                    for (uint32_t m = alive; m; m &= m - 1) {
                        const int cl = __ffs((int)m) - 1;
                        const uint32_t kk = keys[pm_key_at(cl, threadIdx.x)];
                        const float4 dj = sdir[cell_row(cl, kk & 7u)];
                        if (fabsf(dj.x * ds.x + dj.y * ds.y + dj.z * ds.z) >= kStartSepCos) alive &= ~(1u << cl);
                        else if (kk > bk) { bk = kk; bcell = cl; }
                    }
                }
            }
            __syncwarp();  // the key rows are restaged by the next voxel block
            // up to kPreIters Newton steps from every start in turn, then up to
            // kNewtonIters on the best: one inlined copy of the step serves all
            // of them (a small kernel body stays in the instruction cache)
            if (F > 0.f) {
                uint32_t rows = 0u;  // start rows, 7 bits each
                int ns = 0;
    #pragma unroll
                for (int s = 0; s < kStarts; s++)
                    if (live[s]) { rows |= (uint32_t)sj[s] << (7 * s); ns = s + 1; }
                float bA[6], A[6];
                const float4 d0 = sdir[rows & 127u];
                float ux = d0.x, uy = d0.y, uz = d0.z;
                float p = form_at<N>(c, ux, uy, uz, A);
                best = -INFINITY;
                int s = 0;
    #pragma unroll 1
                for (;;) {
                    const bool final_polish = s == ns;
                    polish<N>(c, F, ux, uy, uz, p, A, final_polish ? kNewtonIters : kPreIters);
                    if (final_polish) break;
                    if (p > best) {
                        best = p; bx = ux; by = uy; bz = uz;
    #pragma unroll
                        for (int i = 0; i < 6; i++) bA[i] = A[i];
                    }
                    if (++s < ns) {
                        const float4 d = sdir[(rows >> (7 * s)) & 127u];
                        ux = d.x; uy = d.y; uz = d.z;
                        p = form_at<N>(c, ux, uy, uz, A);
                    } else {
                        ux = bx; uy = by; uz = bz; p = best;
    #pragma unroll
                        for (int i = 0; i < 6; i++) A[i] = bA[i];
                    }
                }
                best = p; bx = ux; by = uy; bz = uz;
            }
        }
        // canonical half-sphere: last non-zero of (z, y, x) positive
        if (bz < 0.f || (bz == 0.f && (by < 0.f || (by == 0.f && bx < 0.f)))) { bx = -bx; by = -by; bz = -bz; }
        if (ok) {
            score[vo] = best;
            orient[vo] = bx;
            orient[Vo + vo] = by;
            orient[2 * Vo + vo] = bz;
            if (frob) frob[vo] = F;
        }
    }
}

// Learned maximiser: the MLP (BF16 tensor cores) predicts the maximising
// direction from C / ||C||_F and Newton polishes it. The plain maximiser's
// probe directions then serve as the check. Their values come from the
// same FP16 tensor-core product as in the plain maximiser (best, its index,
// runner-up); with |x_k| <= 1 and sum mult x^2 = 1, Cauchy-Schwarz bounds
// every FP16 probe value's error by kProbeErr ||C||_F, so every probe is
// below B = max(p(best probe) in FP32, (runner-up + kProbeErr) ||C||_F).
// Where the polished value is below B, a second polish starts from the best
// probe and the better of the two is kept. A voxel is accepted when its
// kept polish converged, its value is not below B (up to 1e-5 ||C||_F), the
// plain maximiser would start from the best probe alone (a second sweep of
// the probe product finds no probe farther than kStartSepDeg from it within
// kStartMargin, by the same FP16 values and test) and the polished direction
// lies within kStartSepDeg of that probe; the others are appended to `list`
// (warp-aggregated atomics) for the plain maximiser, and past the list's
// capacity their score is set to NaN for a sweep instead.
constexpr int kMlThreads = 256;
constexpr int kMlWarps = kMlThreads / 32;

// bound on |FP16 probe value - exact| / ||C||_F: two FP16 roundings of the
// operands (2 * 2^-11 on a sum of |phi x| <= 1) plus subnormal inputs and
// FP32 accumulation, with margin
constexpr float kProbeErr = 1.5e-3f;

template <int N>
__host__ __device__ constexpr size_t ml_smem_bytes()
{
    return kMlpImageBytes + sizeof(__nv_bfloat16) * kMlWarps * 32 * kW1S + sizeof(float) * kMlWarps * 32 * 4 +
           sizeof(__half) * kProbes * pm_kxs(N) + sizeof(float4) * kProbes;
}

template <int N>
__global__ void __launch_bounds__(kMlThreads, 2)
k_peakmap_mlp(const float* __restrict__ C, int64_t V, float* __restrict__ score, float* __restrict__ orient,
              float* __restrict__ frob, const unsigned char* __restrict__ image, ProbeTables tabs,
              uint32_t* __restrict__ list, unsigned long long* __restrict__ count, int64_t cap)
{
    constexpr int K = ncomp3(N);
    constexpr int KP = kpad(N);
    constexpr int KX = mlp_kx(K);
    constexpr int KXS = pm_kxs(N);
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* img = smem;
    size_t off = kMlpImageBytes;
    __nv_bfloat16* sx = reinterpret_cast<__nv_bfloat16*>(smem + off) + (threadIdx.x >> 5) * 32 * kW1S;
    off += sizeof(__nv_bfloat16) * kMlWarps * 32 * kW1S;
    float* sy = reinterpret_cast<float*>(smem + off) + (threadIdx.x >> 5) * 32 * 4;
    off += sizeof(float) * kMlWarps * 32 * 4;
    __half* phih = reinterpret_cast<__half*>(smem + off);
    off += sizeof(__half) * kProbes * KXS;
    float4* sdir = reinterpret_cast<float4*>(smem + off);
    mlp_image_to_smem(image, img);
    {
        const __half* ph = N == 2 ? tabs.phi2h : (N == 4 ? tabs.phi4h : tabs.phi6h);
        const uint4* src = reinterpret_cast<const uint4*>(ph);
        uint4* dst = reinterpret_cast<uint4*>(phih);
        for (int i = threadIdx.x; i < kProbes * KXS / 8; i += blockDim.x) dst[i] = src[i];
        for (int i = threadIdx.x; i < kProbes; i += blockDim.x) sdir[i] = tabs.dir[i];
    }
    __syncthreads();
    const float* phi32 = N == 2 ? tabs.phi2 : (N == 4 ? tabs.phi4 : tabs.phi6);
    const float* b3 = reinterpret_cast<const float*>(img + kMlpOffB3);
    const int lane = threadIdx.x & 31;
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
                for (int b = N - a; b >= 0; b--) {
                    const int cc = N - a - b;
                    const float mult = factf(N) / (factf(a) * factf(b) * factf(cc));
                    c[k] = ok ? __ldg(C + (int64_t)k * V + v) : 0.f;
                    F2 += mult * c[k] * c[k];
                    k++;
                }
#pragma unroll
            for (int k2 = K; k2 < KP; k2++) c[k2] = 0.f;
        }
        const float F = sqrtf(F2);
        const float inv = F > 0.f ? 1.f / F : 0.f;
        // probe values / ||C||_F on the tensor cores: x in FP16 in the staging
        // rows, m16n8k16 with the FP16 probe table, FP32 accumulation; only
        // the best value, its probe and the runner-up are kept
        float pm1 = -INFINITY, pm2 = -INFINITY, pfar = -INFINITY;
        int pj1 = 0;
        {
            __half* hx = reinterpret_cast<__half*>(sx);
#pragma unroll
            for (int k = 0; k < KX; k += 2)
                *reinterpret_cast<__half2*>(hx + lane * kW1S + k) =
                    __floats2half2_rn(k < K ? c[k] * inv : 0.f, k + 1 < K ? c[k + 1] * inv : 0.f);
            __syncwarp();
            const int g = lane >> 2, t = lane & 3;
#pragma unroll 1
            for (int mt = 0; mt < 2; mt++) {
                const __half* r0 = hx + (16 * mt + g) * kW1S + 2 * t;
                const __half* r1 = r0 + 8 * kW1S;
                uint32_t a[KX / 16][4];
#pragma unroll
                for (int ks = 0; ks < KX / 16; ks++) {
                    a[ks][0] = *reinterpret_cast<const uint32_t*>(r0 + 16 * ks);
                    a[ks][1] = *reinterpret_cast<const uint32_t*>(r1 + 16 * ks);
                    a[ks][2] = *reinterpret_cast<const uint32_t*>(r0 + 16 * ks + 8);
                    a[ks][3] = *reinterpret_cast<const uint32_t*>(r1 + 16 * ks + 8);
                }
                float aM = -INFINITY, aS = -INFINITY, bM = -INFINITY, bS = -INFINITY;
                int aI = 0, bI = 0;
                auto upd = [](float v, int j, float& M, float& S, int& I) {
                    if (v > M) { S = M; M = v; I = j; }
                    else if (v > S) S = v;
                };
#pragma unroll 2
                for (int nt = 0; nt < kProbes / 8; nt++) {
                    float acc[4] = {0.f, 0.f, 0.f, 0.f};
                    const __half* br = phih + (nt * 8 + g) * KXS + 2 * t;
#pragma unroll
                    for (int ks = 0; ks < KX / 16; ks++)
                        mma_f16(acc, a[ks], *reinterpret_cast<const uint32_t*>(br + 16 * ks),
                                *reinterpret_cast<const uint32_t*>(br + 16 * ks + 8));
                    const int j0 = nt * 8 + 2 * t;
                    upd(acc[0], j0, aM, aS, aI);
                    upd(acc[1], j0 + 1, aM, aS, aI);
                    upd(acc[2], j0, bM, bS, bI);
                    upd(acc[3], j0 + 1, bM, bS, bI);
                }
                auto merge = [](float& M, float& S, int& I, float oM, float oS, int oI) {
                    if (oM > M || (oM == M && oI < I)) { S = fmaxf(M, fmaxf(S, oS)); M = oM; I = oI; }
                    else S = fmaxf(oM, fmaxf(S, oS));
                };
#pragma unroll
                for (int o = 1; o <= 2; o <<= 1) {
                    merge(aM, aS, aI, __shfl_xor_sync(0xffffffffu, aM, o), __shfl_xor_sync(0xffffffffu, aS, o),
                          __shfl_xor_sync(0xffffffffu, aI, o));
                    merge(bM, bS, bI, __shfl_xor_sync(0xffffffffu, bM, o), __shfl_xor_sync(0xffffffffu, bS, o),
                          __shfl_xor_sync(0xffffffffu, bI, o));
                }
                // second sweep: the best FP16-rounded value among the probes
                // farther than kStartSepDeg from each row's best probe (the
                // plain maximiser's test for a second start)
                const uint4 fa = __ldg(tabs.far + aI), fb = __ldg(tabs.far + bI);
                const uint32_t fwa[4] = {fa.x, fa.y, fa.z, fa.w}, fwb[4] = {fb.x, fb.y, fb.z, fb.w};
                float aF = -INFINITY, bF = -INFINITY;
#pragma unroll
                for (int nt = 0; nt < kProbes / 8; nt++) {
                    float acc[4] = {0.f, 0.f, 0.f, 0.f};
                    const __half* br = phih + (nt * 8 + g) * KXS + 2 * t;
#pragma unroll
                    for (int ks = 0; ks < KX / 16; ks++)
                        mma_f16(acc, a[ks], *reinterpret_cast<const uint32_t*>(br + 16 * ks),
                                *reinterpret_cast<const uint32_t*>(br + 16 * ks + 8));
                    const int j0 = nt * 8 + 2 * t;
                    const uint32_t wa = fwa[nt >> 2] >> (j0 & 31), wb = fwb[nt >> 2] >> (j0 & 31);
                    if (wa & 1u) aF = fmaxf(aF, __half2float(__float2half_rn(acc[0])));
                    if (wa & 2u) aF = fmaxf(aF, __half2float(__float2half_rn(acc[1])));
                    if (wb & 1u) bF = fmaxf(bF, __half2float(__float2half_rn(acc[2])));
                    if (wb & 2u) bF = fmaxf(bF, __half2float(__float2half_rn(acc[3])));
                }
#pragma unroll
                for (int o = 1; o <= 2; o <<= 1) {
                    aF = fmaxf(aF, __shfl_xor_sync(0xffffffffu, aF, o));
                    bF = fmaxf(bF, __shfl_xor_sync(0xffffffffu, bF, o));
                }
                const int r = lane - 16 * mt;
                const int src = 4 * (r & 7);
                const float vM = __shfl_sync(0xffffffffu, r < 8 ? aM : bM, src);
                const float vS = __shfl_sync(0xffffffffu, r < 8 ? aS : bS, src);
                const int vI = __shfl_sync(0xffffffffu, r < 8 ? aI : bI, src);
                const float vF = __shfl_sync(0xffffffffu, r < 8 ? aF : bF, src);
                if (r >= 0 && r < 16) { pm1 = vM; pm2 = vS; pj1 = vI; pfar = vF; }
            }
            __syncwarp();
        }
        // MLP input row (C / ||C||_F in BF16, zero padded to KX columns)
#pragma unroll
        for (int k = 0; k < KX; k += 2) {
            const float x0 = k < K ? c[k] * inv : 0.f;
            const float x1 = k + 1 < K ? c[k + 1] * inv : 0.f;
            *reinterpret_cast<uint32_t*>(sx + lane * kW1S + k) = pack_bf16(x0, x1);
        }
        __syncwarp();
        mlp_warp_bf16<KX>(sx, img, sy);
        __syncwarp();
        float ux = sy[lane * 4] + b3[0], uy = sy[lane * 4 + 1] + b3[1], uz = sy[lane * 4 + 2] + b3[2];
        float best = 0.f;
        bool accept = true;
        if (F > 0.f) {
            const float yn = ux * ux + uy * uy + uz * uz;
            if (yn > 0.f) normalise3(ux, uy, uz);
            else { ux = 0.f; uy = 0.f; uz = 1.f; }
            float A[6];
            best = form_at<N>(c, ux, uy, uz, A);
            bool conv = polish<N>(c, F, ux, uy, uz, best, A, kNewtonIters);
            // bound on every probe value: the best probe in FP32, the others
            // by the runner-up plus the FP16 error bound
            float pexact = 0.f;
            {
                const float4* ph = reinterpret_cast<const float4*>(phi32 + pj1 * KP);
#pragma unroll
                for (int q = 0; q < KP / 4; q++) {
                    const float4 f = __ldg(ph + q);
                    pexact += f.x * c[4 * q] + f.y * c[4 * q + 1] + f.z * c[4 * q + 2] + f.w * c[4 * q + 3];
                }
            }
            const float pm = fmaxf(pexact, (pm2 + kProbeErr) * F);
            const float tol = 1e-5f * F;
            if (!(conv && best >= pm - tol)) {
                const float4 d = sdir[pj1];
                float vx = d.x, vy = d.y, vz = d.z, A2[6];
                float p2 = form_at<N>(c, vx, vy, vz, A2);
                const bool conv2 = polish<N>(c, F, vx, vy, vz, p2, A2, kNewtonIters);
                if (p2 > best) { best = p2; ux = vx; uy = vy; uz = vz; conv = conv2; }
            }
            // accepted only where the plain maximiser would itself use the
            // best probe as its single start (no far probe within the margin)
            // and the polished direction lies in that probe's region, so the
            // two forms end at the same maximum; elsewhere the plain
            // maximiser decides
            const float4 dj = sdir[pj1];
            const bool single = !(pfar >= pm1 - kStartMargin);
            const bool aligned = fabsf(ux * dj.x + uy * dj.y + uz * dj.z) >= kStartSepCos;
            accept = conv && best >= pm - tol && single && aligned;
        } else {
            ux = 0.f; uy = 0.f; uz = 1.f;
        }
        if (uz < 0.f || (uz == 0.f && (uy < 0.f || (uy == 0.f && ux < 0.f)))) { ux = -ux; uy = -uy; uz = -uz; }
        const bool reject = ok && !accept;
        const unsigned rmask = __ballot_sync(0xffffffffu, reject);
        if (rmask) {
            const int leader = __ffs(rmask) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(rmask));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (reject) {
                const unsigned long long pos = base + __popc(rmask & ((1u << lane) - 1u));
                if ((int64_t)pos < cap) list[pos] = (uint32_t)v;
                else score[v] = __int_as_float(0x7fc00000);
            }
        }
        if (ok) {
            if (accept) {
                score[v] = best;
                orient[v] = ux;
                orient[V + v] = uy;
                orient[2 * V + v] = uz;
            }
            if (frob) frob[v] = F;
        }
    }
}

// ---------------------------------------------------------------- host --

// probe directions (spherical Fibonacci on the half-sphere z > 0) and the
// multiplicity-weighted monomials of each order, padded to float4 rows. The
// probes are grouped into kCells cells of 8 neighbours (each cell the
// lowest-index unassigned probe and its 7 nearest unassigned ones, by
// |d . d'|), member m of cell c stored at row cell_row(c, m).
void build_probe_tables(std::vector<float>& out, size_t off[5])
{
    const double ga = M_PI * (3.0 - std::sqrt(5.0));
    std::vector<double> d0(3 * kProbes);
    for (int i = 0; i < kProbes; i++) {
        double z = (i + 0.5) / kProbes, r = std::sqrt(1.0 - z * z), ph = ga * i;
        d0[3 * i] = r * std::cos(ph);
        d0[3 * i + 1] = r * std::sin(ph);
        d0[3 * i + 2] = z;
    }
    std::vector<int> order;
    std::vector<char> used(kProbes, 0);
    for (int seed = 0; seed < kProbes; seed++) {
        if (used[seed]) continue;
        std::vector<std::pair<double, int>> cand;
        for (int j = 0; j < kProbes; j++)
            if (!used[j])
                cand.push_back({-std::fabs(d0[3 * seed] * d0[3 * j] + d0[3 * seed + 1] * d0[3 * j + 1] +
                                           d0[3 * seed + 2] * d0[3 * j + 2]),
                                j});
        std::sort(cand.begin(), cand.end());
        for (int m = 0; m < 8 && m < (int)cand.size(); m++) {
            order.push_back(cand[m].second);
            used[cand[m].second] = 1;
        }
    }
    std::vector<double> d(3 * kProbes);
    for (int c = 0; c < kCells; c++)
        for (int m = 0; m < 8; m++) {
            const int row = cell_row(c, m), j = order[8 * c + m];
            for (int k = 0; k < 3; k++) d[3 * row + k] = d0[3 * j + k];
        }
    out.clear();
    off[0] = 0;
    for (int i = 0; i < kProbes; i++) {
        out.push_back((float)d[3 * i]); out.push_back((float)d[3 * i + 1]);
        out.push_back((float)d[3 * i + 2]); out.push_back(0.f);
    }
    int slot = 1;
    for (int n : {2, 4, 6}) {
        off[slot++] = out.size();
        const int K = ncomp3(n), KP = kpad(n);
        for (int j = 0; j < kProbes; j++) {
            int k = 0;
            for (int a = n; a >= 0; a--)
                for (int b = n - a; b >= 0; b--, k++) {
                    int c = n - a - b;
                    double mult = std::tgamma(n + 1.0) / (std::tgamma(a + 1.0) * std::tgamma(b + 1.0) * std::tgamma(c + 1.0));
                    out.push_back((float)(mult * std::pow(d[3 * j], a) * std::pow(d[3 * j + 1], b) * std::pow(d[3 * j + 2], c)));
                }
            for (; k < KP; k++) out.push_back(0.f);
            (void)K;
        }
    }
    // "far" rows: bit j of row i is set when |d_i . d_j| < cos(kStartSepDeg)
    // (u and -u are the same direction), 4 words per probe
    off[4] = out.size();
    const double cmax = std::cos(kStartSepDeg * M_PI / 180.0);
    std::vector<uint32_t> far(kProbes * 4, 0u);
    for (int i = 0; i < kProbes; i++)
        for (int j = 0; j < kProbes; j++) {
            const double dot = std::fabs(d[3 * i] * d[3 * j] + d[3 * i + 1] * d[3 * j + 1] + d[3 * i + 2] * d[3 * j + 2]);
            if (dot < cmax) far[i * 4 + j / 32] |= 1u << (j % 32);
        }
    out.resize(out.size() + far.size(), 0.f);
    std::memcpy(&out[off[4]], far.data(), far.size() * sizeof(uint32_t));
}

// FP16 copy of a weighted-monomial table: [kProbes][KP] FP32 -> [kProbes][KXS]
__global__ void k_phi_half(const float* __restrict__ phi, int KP, int K, int KXS, __half* __restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kProbes * KXS; i += gridDim.x * blockDim.x) {
        const int j = i / KXS, k = i - j * KXS;
        out[i] = __float2half_rn(k < K ? phi[j * KP + k] : 0.f);
    }
}

void upload_probe_tables(ttm_ctx* ctx)
{
    std::vector<float> h;
    size_t off[5];
    build_probe_tables(h, off);
    ctx->probe_tables.alloc(h.size() * sizeof(float));
    TTM_CUDA_TRY(cudaMemcpy(ctx->probe_tables.p, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
    for (int i = 0; i < 5; i++) ctx->probe_off[i] = off[i];
    size_t total = 0;
    const int orders[3] = {2, 4, 6};
    for (int q = 0; q < 3; q++) {
        ctx->probe_half_off[q] = total;
        total += (size_t)kProbes * pm_kxs(orders[q]);
    }
    ctx->probe_half.alloc(total * sizeof(__half));
    for (int q = 0; q < 3; q++) {
        const int n = orders[q];
        k_phi_half<<<64, 256>>>(ctx->probe_tables.as<float>() + off[1 + q], kpad(n), ncomp3(n), pm_kxs(n),
                                ctx->probe_half.as<__half>() + ctx->probe_half_off[q]);
        TTM_LAUNCH_CHECK();
    }
    TTM_CUDA_TRY(cudaDeviceSynchronize());
}

static ProbeTables probe_tables(ttm_ctx* ctx)
{
    const float* base = ctx->probe_tables.as<float>();
    const __half* hb = ctx->probe_half.as<__half>();
    return ProbeTables{reinterpret_cast<const float4*>(base + ctx->probe_off[0]), base + ctx->probe_off[1],
                       base + ctx->probe_off[2], base + ctx->probe_off[3],
                       reinterpret_cast<const uint4*>(base + ctx->probe_off[4]),
                       hb + ctx->probe_half_off[0], hb + ctx->probe_half_off[1], hb + ctx->probe_half_off[2]};
}

// plain maximiser over all voxels (PM_ALL) or the learned path's fallbacks
static void plain_run(ttm_ctx* ctx, int n, const float* C, int64_t V, float* score, float* orient, float* frob,
                      const PmGeom& geo, cudaStream_t st)
{
    const ProbeTables t = probe_tables(ctx);
    const int64_t items = geo.mode == PM_BOX ? (int64_t)geo.bz * geo.by * geo.bx : V;
    const int64_t blocks = std::max<int64_t>(1, ceil_div(items, kPmThreads));
    const size_t smem = pm_smem_bytes(n);
    // enough CTAs to fill every SM several times, then a grid stride
    const int64_t grid = std::min<int64_t>(blocks, (int64_t)ctx->num_sms * 32);
    // static tables + dynamic probe values can exceed the default 48 KB
    // total, so the dynamic size is always declared
#define TTM_PM_LAUNCH(N_)                                                                          \
    TTM_CUDA_TRY(cudaFuncSetAttribute(k_peakmap<N_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    k_peakmap<N_><<<(unsigned)grid, kPmThreads, smem, st>>>(C, V, score, orient, frob, t, geo);
    switch (n) {
        case 2: TTM_PM_LAUNCH(2); break;
        case 4: TTM_PM_LAUNCH(4); break;
        case 6: TTM_PM_LAUNCH(6); break;
        default: throw Error{E_UNSUPPORTED, "order must be 2, 4 or 6"};
    }
#undef TTM_PM_LAUNCH
    TTM_LAUNCH_CHECK();
}

void peakmap_run(ttm_ctx* ctx, int n, const float* C, int64_t V, float* score, float* orient, float* frob,
                 cudaStream_t st)
{
    plain_run(ctx, n, C, V, score, orient, frob, PmGeom(), st);
}

// plain maximiser over box b (z0, z1, y0, y1, x0, x1) of C on a Z x Yin x
// Xin grid, maps written on a Zo x Yout x Xout grid at the same coordinates
void peakmap_box_run(ttm_ctx* ctx, int n, const float* C, int Z, int Yin, int Xin, const int* b, int Zo, int Yout,
                     int Xout, float* score, float* orient, float* frob, cudaStream_t st)
{
    PmGeom g;
    g.mode = PM_BOX;
    g.z0 = b[0]; g.y0 = b[2]; g.x0 = b[4];
    g.bz = b[1] - b[0]; g.by = b[3] - b[2]; g.bx = b[5] - b[4];
    g.Yin = Yin; g.Xin = Xin; g.Yout = Yout; g.Xout = Xout;
    g.Vout = (int64_t)Zo * Yout * Xout;
    if (g.bz <= 0 || g.by <= 0 || g.bx <= 0) return;
    plain_run(ctx, n, C, (int64_t)Z * Yin * Xin, score, orient, frob, g, st);
}

// learned maximiser, then the plain one on its rejected voxels
static void peakmap_learned_run(ttm_plan* P, ttm_mlp* M, const float* C, int64_t V, float* score, float* orient,
                                float* frob, cudaStream_t st)
{
    ttm_ctx* ctx = P->ctx;
    const int n = P->fp.order_n;
    uint32_t* list = P->cand.as<uint32_t>();
    const int64_t cap = (int64_t)(P->cand.bytes / sizeof(uint32_t));
    unsigned long long* count = P->fb_count.as<unsigned long long>();
    const ProbeTables tabs = probe_tables(ctx);
    TTM_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(unsigned long long), st));
    const int64_t blocks = ceil_div(V, kMlThreads);
    const int64_t grid = std::min<int64_t>(blocks, (int64_t)ctx->num_sms * 2);
#define TTM_ML_LAUNCH(N_)                                                                                         \
    {                                                                                                              \
        const size_t smem = ml_smem_bytes<N_>();                                                                   \
        TTM_CUDA_TRY(cudaFuncSetAttribute(k_peakmap_mlp<N_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        k_peakmap_mlp<N_><<<(unsigned)grid, kMlThreads, smem, st>>>(C, V, score, orient, frob,                     \
                                                                   M->image.as<unsigned char>(), tabs, list,      \
                                                                   count, cap);                                   \
    }
    switch (n) {
        case 2: TTM_ML_LAUNCH(2); break;
        case 4: TTM_ML_LAUNCH(4); break;
        case 6: TTM_ML_LAUNCH(6); break;
        default: throw Error{E_UNSUPPORTED, "order must be 2, 4 or 6"};
    }
#undef TTM_ML_LAUNCH
    TTM_LAUNCH_CHECK();
    PmGeom g;
    g.list = list;
    g.list_count = count;
    g.list_cap = cap;
    g.mode = PM_LIST;
    plain_run(ctx, n, C, V, score, orient, frob, g, st);
    g.mode = PM_SWEEP;
    plain_run(ctx, n, C, V, score, orient, frob, g, st);
}

}  // namespace ttm

using namespace ttm;

extern "C" ttm_status ttm_peak_map(ttm_plan* plan, const float* d_C, ttm_maximiser mode, const ttm_mlp* mlp,
                                   float* d_score, float* d_orient, float* d_frob, void* stream)
{
    if (!plan) return TTM_E_INVALID_ARG;
    try {
        TTM_REQUIRE(d_C && d_score && d_orient, E_INVALID_ARG, "null pointer argument");
        TTM_REQUIRE(mode == TTM_MAX_PLAIN || mode == TTM_MAX_MLP_WARM, E_INVALID_ARG, "unknown maximiser");
        TTM_REQUIRE(mode == TTM_MAX_MLP_WARM || mlp == nullptr, E_INVALID_ARG,
                    "mlp must be NULL for the plain maximiser");
        TTM_REQUIRE(mode == TTM_MAX_PLAIN || mlp != nullptr, E_INVALID_ARG, "the learned maximiser needs an mlp");
        TTM_REQUIRE(plan->fp.dprime == 3 || mode == TTM_MAX_PLAIN, E_UNSUPPORTED,
                    "the learned maximiser works on the 2-sphere (d' = 3)");
        TTM_CUDA_TRY(cudaSetDevice(plan->ctx->device));
        const Prep& p = plan->prep;
        const int64_t V = (int64_t)p.Z * p.Y * p.X;
        cudaStream_t st = (cudaStream_t)stream;
        if (plan->fp.dprime == 4) {
            stage_begin(plan, st);
            peakmap4_run(plan->ctx, plan->fp.order_n, d_C, V, d_score, d_orient, d_frob, st);
            stage_end(plan, ST_PEAKMAP, st);
        } else if (mode == TTM_MAX_MLP_WARM) {
            ttm_mlp* M = const_cast<ttm_mlp*>(mlp);
            TTM_REQUIRE(M->K == plan->K, E_INVALID_ARG, "mlp input count differs from the plan's component count");
            TTM_REQUIRE(M->ctx->device == plan->ctx->device, E_INVALID_ARG, "mlp lives on another device");
            TTM_REQUIRE(V <= (int64_t)UINT32_MAX, E_SHAPE, "the learned maximiser indexes voxels with 32 bits");
            mlp_refresh_image(M);
            stage_begin(plan, st);
            peakmap_learned_run(plan, M, d_C, V, d_score, d_orient, d_frob, st);
            stage_end(plan, ST_PEAKMAP, st);
        } else {
            stage_begin(plan, st);
            peakmap_run(plan->ctx, plan->fp.order_n, d_C, V, d_score, d_orient, d_frob, st);
            stage_end(plan, ST_PEAKMAP, st);
        }
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(plan->ctx, e);
    }
}

extern "C" ttm_status ttm_plan_fallback_count(ttm_plan* plan, int64_t* h_count, void* stream)
{
    if (!plan || !h_count) return TTM_E_INVALID_ARG;
    try {
        TTM_CUDA_TRY(cudaSetDevice(plan->ctx->device));
        unsigned long long n = 0;
        cudaStream_t st = (cudaStream_t)stream;
        TTM_CUDA_TRY(cudaMemcpyAsync(&n, plan->fb_count.p, sizeof(n), cudaMemcpyDeviceToHost, st));
        TTM_CUDA_TRY(cudaStreamSynchronize(st));
        *h_count = (int64_t)n;
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(plan->ctx, e);
    }
}
