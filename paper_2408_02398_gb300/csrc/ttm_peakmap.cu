// ttm_peakmap.cu -- per-voxel contraction and maximisation over unit
// directions (Sec. 3.1 and 3.2):
//   F(x) = ||C(x)||_F,  s(x) = max_{|u|=1} p_x(u),  u*(x) = argmax,
//   p_x(u) = C(x) . u^{(x)n} = sum_alpha mult(alpha) C_alpha(x) u^alpha.
//
// One thread per voxel, components loaded structure-of-arrays (coalesced).
// The form is evaluated at P fixed probe directions on the half-sphere
// (p is even); the probes whose value is not below any of their nearest
// probes (discrete local maxima) are the candidate basins, and the best
// NS of them are polished by Riemannian Newton steps on the sphere, with a
// shifted power step (SS-HOPM, shift (n-1)||C||_F) whenever Newton does not
// apply or does not increase p.
#include <cmath>
#include <vector>

#include "ttm_internal.h"

namespace ttm {

constexpr int kProbes = 96;
constexpr int kProbeNbr = 6;
constexpr int kPmThreads = 128;
constexpr int kStarts = 3;
constexpr int kNewtonIters = 16;

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

// p, gradient and (optionally) Hessian of sum_k cm_k x^a y^b z^c, with cm
// the multiplicity-weighted components (graded-lex descending exponents)
template <int N, bool HESS>
__device__ __forceinline__ void form3(const float* cm, float ux, float uy, float uz, float& p, float* g, float* H)
{
    float px[N + 1], py[N + 1], pz[N + 1];
    px[0] = py[0] = pz[0] = 1.f;
#pragma unroll
    for (int e = 1; e <= N; e++) { px[e] = px[e - 1] * ux; py[e] = py[e - 1] * uy; pz[e] = pz[e - 1] * uz; }
    p = 0.f;
    g[0] = g[1] = g[2] = 0.f;
    if (HESS) { H[0] = H[1] = H[2] = H[3] = H[4] = H[5] = 0.f; }
    int k = 0;
#pragma unroll
    for (int a = N; a >= 0; a--) {
#pragma unroll
        for (int b = N - a; b >= 0; b--) {
            const int c = N - a - b;
            const float w = cm[k++];
            p += w * px[a] * py[b] * pz[c];
            if (a > 0) g[0] += w * a * px[a - 1] * py[b] * pz[c];
            if (b > 0) g[1] += w * b * px[a] * py[b - 1] * pz[c];
            if (c > 0) g[2] += w * c * px[a] * py[b] * pz[c - 1];
            if (HESS) {
                if (a > 1) H[0] += w * a * (a - 1) * px[a - 2] * py[b] * pz[c];
                if (a > 0 && b > 0) H[1] += w * a * b * px[a - 1] * py[b - 1] * pz[c];
                if (a > 0 && c > 0) H[2] += w * a * c * px[a - 1] * py[b] * pz[c - 1];
                if (b > 1) H[3] += w * b * (b - 1) * px[a] * py[b - 2] * pz[c];
                if (b > 0 && c > 0) H[4] += w * b * c * px[a] * py[b - 1] * pz[c - 1];
                if (c > 1) H[5] += w * c * (c - 1) * px[a] * py[b] * pz[c - 2];
            }
        }
    }
}

template <int N>
__device__ __forceinline__ float form_value(const float* cm, float ux, float uy, float uz)
{
    float p, g[3], H[6];
    form3<N, false>(cm, ux, uy, uz, p, g, H);
    return p;
}

__device__ __forceinline__ void normalise3(float& x, float& y, float& z)
{
    float s = rsqrtf(x * x + y * y + z * z);
    x *= s; y *= s; z *= s;
}

// polish u to a local maximum; returns p(u)
template <int N>
__device__ float polish(const float* cm, float frob, float& ux, float& uy, float& uz)
{
    const float shift = (N - 1) * frob;
    const float tol_g = 1e-6f * frob;
    float p = 0.f;
    for (int it = 0; it < kNewtonIters; it++) {
        float g[3], H[6];
        form3<N, true>(cm, ux, uy, uz, p, g, H);
        const float u[3] = {ux, uy, uz};
        const float lam = ux * g[0] + uy * g[1] + uz * g[2];
        // tangent basis from the Householder reflection mapping e_k to -+u
        int kmax = 0;
        if (fabsf(uy) > fabsf(u[kmax])) kmax = 1;
        if (fabsf(uz) > fabsf(u[kmax])) kmax = 2;
        float v[3] = {ux, uy, uz};
        v[kmax] += u[kmax] >= 0.f ? 1.f : -1.f;
        const float vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        float B[2][3];
        int nb = 0;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            if (j == kmax) continue;
#pragma unroll
            for (int i = 0; i < 3; i++) B[nb][i] = (i == j ? 1.f : 0.f) - 2.f * v[i] * v[j] / vv;
            nb++;
        }
        float gr[2], Hb[2][3];
#pragma unroll
        for (int a = 0; a < 2; a++) {
            gr[a] = B[a][0] * g[0] + B[a][1] * g[1] + B[a][2] * g[2];
            Hb[a][0] = H[0] * B[a][0] + H[1] * B[a][1] + H[2] * B[a][2];
            Hb[a][1] = H[1] * B[a][0] + H[3] * B[a][1] + H[4] * B[a][2];
            Hb[a][2] = H[2] * B[a][0] + H[4] * B[a][1] + H[5] * B[a][2];
        }
        if (sqrtf(gr[0] * gr[0] + gr[1] * gr[1]) <= tol_g) break;
        // negated Riemannian Hessian in the basis
        float h00 = -(B[0][0] * Hb[0][0] + B[0][1] * Hb[0][1] + B[0][2] * Hb[0][2] - lam);
        float h01 = -(B[1][0] * Hb[0][0] + B[1][1] * Hb[0][1] + B[1][2] * Hb[0][2]);
        float h11 = -(B[1][0] * Hb[1][0] + B[1][1] * Hb[1][1] + B[1][2] * Hb[1][2] - lam);
        float det = h00 * h11 - h01 * h01;
        bool moved = false;
        if (h00 > 0.f && det > 0.f) {
            float x0 = (h11 * gr[0] - h01 * gr[1]) / det;
            float x1 = (h00 * gr[1] - h01 * gr[0]) / det;
            float nx = ux + x0 * B[0][0] + x1 * B[1][0];
            float ny = uy + x0 * B[0][1] + x1 * B[1][1];
            float nz = uz + x0 * B[0][2] + x1 * B[1][2];
            normalise3(nx, ny, nz);
            float pn = form_value<N>(cm, nx, ny, nz);
            if (pn >= p - 1e-7f * frob) { ux = nx; uy = ny; uz = nz; moved = true; }
        }
        if (!moved) {
            // shifted power step: u <- normalise(grad / N + shift u), never decreases p
            float nx = g[0] / N + shift * ux, ny = g[1] / N + shift * uy, nz = g[2] / N + shift * uz;
            normalise3(nx, ny, nz);
            ux = nx; uy = ny; uz = nz;
        }
    }
    return form_value<N>(cm, ux, uy, uz);
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
    float c[K], cm[K];
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
                cm[k] = mult * c[k];
                F2 += mult * c[k] * c[k];
                k++;
            }
    }
    const float F = sqrtf(F2);
    const float* phi = phi_table<N>();
    for (int j = 0; j < kProbes; j++) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < K; k++) acc += phi[j * K + k] * c[k];
        pv[j * kPmThreads + threadIdx.x] = acc;
    }
    // best kStarts discrete local maxima (value desc, probe index asc)
    int sj[kStarts];
    float sv[kStarts];
#pragma unroll
    for (int s = 0; s < kStarts; s++) { sj[s] = -1; sv[s] = -INFINITY; }
    for (int j = 0; j < kProbes; j++) {
        const float pj = pv[j * kPmThreads + threadIdx.x];
        bool is_max = true;
#pragma unroll
        for (int b = 0; b < kProbeNbr; b++)
            if (pv[c_nbr[j * kProbeNbr + b] * kPmThreads + threadIdx.x] > pj) is_max = false;
        if (!is_max || !(pj > sv[kStarts - 1])) continue;
        int pos = kStarts - 1;
        while (pos > 0 && sv[pos - 1] < pj) { sv[pos] = sv[pos - 1]; sj[pos] = sj[pos - 1]; pos--; }
        sv[pos] = pj;
        sj[pos] = j;
    }
    float best = -INFINITY, bx = 0.f, by = 0.f, bz = 1.f;
    for (int s = 0; s < kStarts; s++) {
        if (sj[s] < 0) continue;
        float ux = c_dir[3 * sj[s]], uy = c_dir[3 * sj[s] + 1], uz = c_dir[3 * sj[s] + 2];
        float ps = polish<N>(cm, F, ux, uy, uz);
        if (ps > best) { best = ps; bx = ux; by = uy; bz = uz; }
    }
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
