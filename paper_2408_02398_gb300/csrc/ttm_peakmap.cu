// ttm_peakmap.cu -- per-voxel contraction and maximisation over unit
// directions (Sec. 3.1 and 3.2):
//   F(x) = ||C(x)||_F,  s(x) = max_{|u|=1} p_x(u),  u*(x) = argmax,
//   p_x(u) = C(x) . u^{(x)n} = sum_alpha mult(alpha) C_alpha(x) u^alpha.
//
// One thread per voxel, components loaded structure-of-arrays (coalesced).
// The form is evaluated at P fixed probe directions on the half-sphere
// (p is even); the probes whose value is not below any of their nearest
// probes (discrete local maxima) are the candidate basins, and the best NS
// of them are polished on the sphere. The derivatives come from the
// contraction A = C . u^{n-2} (a symmetric 3x3 matrix): p = u^T A u,
// grad p = n A u, Hess p = n (n-1) A. Each polish step is a Riemannian
// Newton step in a Householder tangent basis, limited to 0.5 rad; where the
// tangent Hessian is not negative definite it is shifted until it is (a
// Levenberg-Marquardt step), the step is halved until p does not decrease,
// and a shifted power step (SS-HOPM, shift (n-1)||C||_F, never decreasing)
// is the last resort.
#include <cmath>
#include <vector>

#include "ttm_internal.h"

namespace ttm {

constexpr int kProbes = 128;
constexpr int kProbeNbr = 6;
constexpr int kPmThreads = 128;
constexpr int kStarts = 4;
constexpr int kNewtonIters = 12;

__constant__ float c_phi2[kProbes * 6];
__constant__ float c_phi4[kProbes * 15];
__constant__ float c_phi6[kProbes * 28];
__constant__ float c_dir[kProbes * 3];
__constant__ unsigned char c_nbr[kProbes * kProbeNbr];

template <int N> __device__ __forceinline__ const float* phi_table();
template <> __device__ __forceinline__ const float* phi_table<2>() { return c_phi2; }
template <> __device__ __forceinline__ const float* phi_table<4>() { return c_phi4; }
template <> __device__ __forceinline__ const float* phi_table<6>() { return c_phi6; }

__host__ __device__ constexpr int ncomp3(int n) { return (n + 1) * (n + 2) / 2; }
__host__ __device__ constexpr float factf(int n) { return n <= 1 ? 1.f : n * factf(n - 1); }
// position of exponents (a, b, n-a-b) in graded-lex descending order
__host__ __device__ constexpr int cidx(int n, int a, int b) { return (n - a) * (n - a + 1) / 2 + (n - a - b); }

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

template <int N>
__device__ __forceinline__ float form_value(const float* c, float ux, float uy, float uz)
{
    float A[6];
    contract2<N>(c, ux, uy, uz, A);
    float ax = A[0] * ux + A[1] * uy + A[2] * uz;
    float ay = A[1] * ux + A[3] * uy + A[4] * uz;
    float az = A[2] * ux + A[4] * uy + A[5] * uz;
    return ux * ax + uy * ay + uz * az;
}

__device__ __forceinline__ void normalise3(float& x, float& y, float& z)
{
    float s = rsqrtf(x * x + y * y + z * z);
    x *= s; y *= s; z *= s;
}

// polish u to a local maximum of p; returns p(u)
template <int N>
__device__ float polish(const float* c, float frob, float& ux, float& uy, float& uz)
{
    const float tol_g2 = 1e-12f * frob * frob;  // |tangent gradient| <= 1e-6 ||C||_F
    const float tol_p = 1e-7f * frob;
    const float hN = (float)(N * (N - 1));
    float p = 0.f;
    for (int it = 0; it < kNewtonIters; it++) {
        float A[6];
        contract2<N>(c, ux, uy, uz, A);
        const float ax = A[0] * ux + A[1] * uy + A[2] * uz;
        const float ay = A[1] * ux + A[3] * uy + A[4] * uz;
        const float az = A[2] * ux + A[4] * uy + A[5] * uz;
        p = ux * ax + uy * ay + uz * az;
        // grad = N A u, Hess = N (N-1) A, u . grad = N p.
        // Tangent basis: the Householder reflection of v = u + sign(u_k) e_k
        // (k = largest |u_k|) maps e_k to -+u; its other two columns
        // b_j = e_j - (2 v_j / v.v) v span the tangent plane.
        const float fx = fabsf(ux), fy = fabsf(uy), fz = fabsf(uz);
        const int kmax = (fx >= fy && fx >= fz) ? 0 : (fy >= fz ? 1 : 2);
        const float vx = ux + (kmax == 0 ? (ux >= 0.f ? 1.f : -1.f) : 0.f);
        const float vy = uy + (kmax == 1 ? (uy >= 0.f ? 1.f : -1.f) : 0.f);
        const float vz = uz + (kmax == 2 ? (uz >= 0.f ? 1.f : -1.f) : 0.f);
        const float r2 = __fdividef(2.f, vx * vx + vy * vy + vz * vz);
        const float vj1 = kmax == 0 ? vy : vx;  // j1 = first index != kmax
        const float vj2 = kmax == 2 ? vy : vz;  // j2 = last index != kmax
        const float b0x = (kmax != 0 ? 1.f : 0.f) - r2 * vj1 * vx;
        const float b0y = (kmax == 0 ? 1.f : 0.f) - r2 * vj1 * vy;
        const float b0z = -r2 * vj1 * vz;
        const float b1x = -r2 * vj2 * vx;
        const float b1y = (kmax == 2 ? 1.f : 0.f) - r2 * vj2 * vy;
        const float b1z = (kmax != 2 ? 1.f : 0.f) - r2 * vj2 * vz;
        const float g0 = N * (b0x * ax + b0y * ay + b0z * az);
        const float g1 = N * (b1x * ax + b1y * ay + b1z * az);
        if (g0 * g0 + g1 * g1 <= tol_g2) break;
        // A b0, A b1
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
        if (lmin <= 1e-6f * frob) { const float sh = 0.05f * frob - lmin; h00 += sh; h11 += sh; }
        const float idet = __frcp_rn(h00 * h11 - h01 * h01);
        float x0 = (h11 * g0 - h01 * g1) * idet;
        float x1 = (h00 * g1 - h01 * g0) * idet;
        const float xn2 = x0 * x0 + x1 * x1;
        if (xn2 > 0.25f) { const float sc = 0.5f * rsqrtf(xn2); x0 *= sc; x1 *= sc; }  // |step| <= 0.5 rad
        const float dx = x0 * b0x + x1 * b1x, dy = x0 * b0y + x1 * b1y, dz = x0 * b0z + x1 * b1z;
        bool moved = false;
        float t = 1.f;
#pragma unroll 1
        for (int bt = 0; bt < 4; bt++, t *= 0.5f) {
            float nx = ux + t * dx, ny = uy + t * dy, nz = uz + t * dz;
            normalise3(nx, ny, nz);
            const float pn = form_value<N>(c, nx, ny, nz);
            if (pn >= p - tol_p) { ux = nx; uy = ny; uz = nz; p = pn; moved = true; break; }
        }
        if (!moved) {
            // shifted power step: u <- normalise(A u + (N-1) ||C||_F u), never decreases p
            const float shift = (N - 1) * frob;
            float nx = ax + shift * ux, ny = ay + shift * uy, nz = az + shift * uz;
            normalise3(nx, ny, nz);
            ux = nx; uy = ny; uz = nz;
        }
    }
    return form_value<N>(c, ux, uy, uz);
}

template <int N>
__global__ void __launch_bounds__(kPmThreads)
k_peakmap(const float* __restrict__ C, int64_t V, float* __restrict__ score, float* __restrict__ orient,
          float* __restrict__ frob)
{
    constexpr int K = ncomp3(N);
    extern __shared__ float pv[];  // [kProbes][kPmThreads]
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = v < V;
    float c[K];
    float F2 = 0.f;
    {
        int k = 0;
#pragma unroll
        for (int a = N; a >= 0; a--)
#pragma unroll
            for (int b = N - a; b >= 0; b--) {
                const int cc = N - a - b;
                const float mult = factf(N) / (factf(a) * factf(b) * factf(cc));
                c[k] = ok ? C[(int64_t)k * V + v] : 0.f;
                F2 += mult * c[k] * c[k];
                k++;
            }
    }
    const float F = sqrtf(F2);
    const float* phi = phi_table<N>();
#pragma unroll 4
    for (int j = 0; j < kProbes; j++) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < K; k++) acc += phi[j * K + k] * c[k];
        pv[j * kPmThreads + threadIdx.x] = acc;
    }
    // best kStarts discrete local maxima (value desc, probe index asc); a
    // probe is examined only if it would enter the list (kept in registers:
    // insertion by unrolled compare-and-swap)
    int sj[kStarts];
    float sv[kStarts];
#pragma unroll
    for (int s = 0; s < kStarts; s++) { sj[s] = -1; sv[s] = -INFINITY; }
    for (int j = 0; j < kProbes; j++) {
        const float pj = pv[j * kPmThreads + threadIdx.x];
        if (!(pj > sv[kStarts - 1])) continue;
        bool is_max = true;
#pragma unroll
        for (int b = 0; b < kProbeNbr; b++)
            if (pv[c_nbr[j * kProbeNbr + b] * kPmThreads + threadIdx.x] > pj) is_max = false;
        if (!is_max) continue;
        float cv = pj;
        int cj = j;
#pragma unroll
        for (int s = 0; s < kStarts; s++) {
            if (cv > sv[s]) {
                const float tv = sv[s]; const int tj = sj[s];
                sv[s] = cv; sj[s] = cj;
                cv = tv; cj = tj;
            }
        }
    }
    float best = -INFINITY, bx = 0.f, by = 0.f, bz = 1.f;
#pragma unroll
    for (int s = 0; s < kStarts; s++) {
        if (sj[s] < 0 || F == 0.f) continue;
        float ux = c_dir[3 * sj[s]], uy = c_dir[3 * sj[s] + 1], uz = c_dir[3 * sj[s] + 2];
        const float ps = polish<N>(c, F, ux, uy, uz);
        if (ps > best) { best = ps; bx = ux; by = uy; bz = uz; }
    }
    if (F == 0.f) best = 0.f;
    // canonical half-sphere: last non-zero of (z, y, x) positive
    if (bz < 0.f || (bz == 0.f && (by < 0.f || (by == 0.f && bx < 0.f)))) { bx = -bx; by = -by; bz = -bz; }
    if (ok) {
        score[v] = best;
        orient[v] = bx;
        orient[V + v] = by;
        orient[2 * V + v] = bz;
        if (frob) frob[v] = F;
    }
}

// ---------------------------------------------------------------- host --

// probe directions (spherical Fibonacci on the half-sphere z > 0), their
// nearest neighbours (u ~ -u) and the weighted monomials per order
void upload_probe_tables()
{
    const double ga = M_PI * (3.0 - std::sqrt(5.0));
    std::vector<double> d(3 * kProbes);
    for (int i = 0; i < kProbes; i++) {
        double z = (i + 0.5) / kProbes, r = std::sqrt(1.0 - z * z), ph = ga * i;
        d[3 * i] = r * std::cos(ph);
        d[3 * i + 1] = r * std::sin(ph);
        d[3 * i + 2] = z;
    }
    std::vector<unsigned char> nb(kProbes * kProbeNbr);
    for (int i = 0; i < kProbes; i++) {
        double bd[kProbeNbr];
        int bi[kProbeNbr], n = 0;
        for (int j = 0; j < kProbes; j++) {
            if (j == i) continue;
            double dot = std::fabs(d[3 * i] * d[3 * j] + d[3 * i + 1] * d[3 * j + 1] + d[3 * i + 2] * d[3 * j + 2]);
            if (n == kProbeNbr && dot <= bd[kProbeNbr - 1]) continue;
            int pos = n < kProbeNbr ? n++ : kProbeNbr - 1;
            while (pos > 0 && bd[pos - 1] < dot) { bd[pos] = bd[pos - 1]; bi[pos] = bi[pos - 1]; pos--; }
            bd[pos] = dot;
            bi[pos] = j;
        }
        for (int b = 0; b < kProbeNbr; b++) nb[i * kProbeNbr + b] = (unsigned char)bi[b];
    }
    std::vector<float> df(d.begin(), d.end());
    TTM_CUDA_TRY(cudaMemcpyToSymbol(c_dir, df.data(), df.size() * sizeof(float)));
    TTM_CUDA_TRY(cudaMemcpyToSymbol(c_nbr, nb.data(), nb.size()));
    for (int n : {2, 4, 6}) {
        std::vector<float> phi;
        for (int j = 0; j < kProbes; j++)
            for (int a = n; a >= 0; a--)
                for (int b = n - a; b >= 0; b--) {
                    int c = n - a - b;
                    double mult = std::tgamma(n + 1.0) / (std::tgamma(a + 1.0) * std::tgamma(b + 1.0) * std::tgamma(c + 1.0));
                    double val = mult * std::pow(d[3 * j], a) * std::pow(d[3 * j + 1], b) * std::pow(d[3 * j + 2], c);
                    phi.push_back((float)val);
                }
        if (n == 2) TTM_CUDA_TRY(cudaMemcpyToSymbol(c_phi2, phi.data(), phi.size() * sizeof(float)));
        if (n == 4) TTM_CUDA_TRY(cudaMemcpyToSymbol(c_phi4, phi.data(), phi.size() * sizeof(float)));
        if (n == 6) TTM_CUDA_TRY(cudaMemcpyToSymbol(c_phi6, phi.data(), phi.size() * sizeof(float)));
    }
}

void peakmap_run(int n, const float* C, int64_t V, float* score, float* orient, float* frob, cudaStream_t st)
{
    const size_t smem = (size_t)kProbes * kPmThreads * sizeof(float);
    const unsigned grid = (unsigned)ceil_div(V, kPmThreads);
    switch (n) {
        case 2: set_smem(k_peakmap<2>, smem); k_peakmap<2><<<grid, kPmThreads, smem, st>>>(C, V, score, orient, frob); break;
        case 4: set_smem(k_peakmap<4>, smem); k_peakmap<4><<<grid, kPmThreads, smem, st>>>(C, V, score, orient, frob); break;
        case 6: set_smem(k_peakmap<6>, smem); k_peakmap<6><<<grid, kPmThreads, smem, st>>>(C, V, score, orient, frob); break;
        default: throw Error{E_UNSUPPORTED, "order must be 2, 4 or 6"};
    }
    TTM_LAUNCH_CHECK();
}

}  // namespace ttm

using namespace ttm;

extern "C" ttm_status ttm_peak_map(ttm_plan* plan, const float* d_C, ttm_maximiser mode, const void* mlp,
                                   float* d_score, float* d_orient, float* d_frob, void* stream)
{
    if (!plan) return TTM_E_INVALID_ARG;
    try {
        TTM_REQUIRE(d_C && d_score && d_orient, E_INVALID_ARG, "null pointer argument");
        TTM_REQUIRE(mode == TTM_MAX_PLAIN, E_UNSUPPORTED, "only the plain maximiser is built in this version");
        TTM_REQUIRE(mlp == nullptr, E_INVALID_ARG, "mlp must be NULL for the plain maximiser");
        TTM_CUDA_TRY(cudaSetDevice(plan->ctx->device));
        const Prep& p = plan->prep;
        const int64_t V = (int64_t)p.Z * p.Y * p.X;
        stage_begin(plan, (cudaStream_t)stream);
        peakmap_run(plan->fp.order_n, d_C, V, d_score, d_orient, d_frob, (cudaStream_t)stream);
        stage_end(plan, ST_PEAKMAP, (cudaStream_t)stream);
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(plan->ctx, e);
    }
}
