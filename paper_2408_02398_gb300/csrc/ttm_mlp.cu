// ttm_mlp.cu -- the learned warm start: an MLP K -> 128 -> 128 -> 3 with
// GELU activations (tanh form) and a normalised output u_hat = y / |y|
// that predicts the maximising direction of the form C . u^{(x)n} from the
// components scaled to unit Frobenius norm. Loss per sample:
// 1 - (u_hat . u*)^2 (independent of the sign of u*).
//
// Training runs on the GPU with the kernels below: a tiled FP32 SGEMM for
// the six matrix products of a forward/backward step, fused bias + GELU,
// the GELU derivative, the normalised-output loss gradient, column sums for
// the bias gradients, and Adam. Parameters are one flat FP32 array:
// W1 [H][K], b1 [H], W2 [H][H], b2 [H], W3 [3][H], b3 [3].
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "mlp_mma.cuh"
#include "ttm_internal.h"

namespace ttm {

constexpr int kH = kMlpH;

__host__ __device__ inline int64_t mlp_num_params(int K) { return (int64_t)kH * K + kH + kH * kH + kH + 3 * kH + 3; }

// ------------------------------------------------------------- kernels --

// C[M][N] (+)= op(A) op(B); op(A)[m][k] = TA ? A[k lda + m] : A[m lda + k],
// op(B)[k][n] = TB ? B[n ldb + k] : B[k ldb + n]. 64 x 64 tiles, 4 x 4 per thread.
template <bool TA, bool TB, bool ACC>
__global__ void __launch_bounds__(256) k_sgemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                               const float* __restrict__ B, int ldb, float* __restrict__ C, int ldc)
{
    __shared__ float As[16][65], Bs[16][65];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = tid; e < 64 * 16; e += 256) {
            const int kk = e / 64, mm = e % 64;
            const int m = m0 + mm, k = k0 + kk;
            float a = 0.f, b = 0.f;
            if (m < M && k < K) a = TA ? A[(int64_t)k * lda + m] : A[(int64_t)m * lda + k];
            const int n = n0 + mm;
            if (n < N && k < K) b = TB ? B[(int64_t)n * ldb + k] : B[(int64_t)k * ldb + n];
            As[kk][mm] = a;
            Bs[kk][mm] = b;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; kk++) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) { a[i] = As[kk][ty * 4 + i]; b[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m < M && n < N) {
                float* c = C + (int64_t)m * ldc + n;
                *c = ACC ? *c + acc[i][j] : acc[i][j];
            }
        }
}

// The same product with op(A) and op(B) rounded to BF16 (nearest even) as
// they are staged and multiplied on the tensor cores (mma.sync m16n8k16,
// FP32 accumulate): the BF16 training mode. 64 x 64 tiles, k steps of 16;
// warp w owns rows 16 (w >> 1) .. +16 and columns 32 (w & 1) .. +32 of the
// tile (four 8-column MMA tiles). Shared rows of 24 BF16 (48 bytes) keep the
// fragment loads of a warp in distinct banks.
template <bool TA, bool TB, bool ACC>
__global__ void __launch_bounds__(256) k_gemm_bf16(int M, int N, int K, const float* __restrict__ A, int lda,
                                                   const float* __restrict__ B, int ldb, float* __restrict__ C,
                                                   int ldc)
{
    __shared__ __align__(16) __nv_bfloat16 As[64][24], Bs[64][24];  // [m][k], [n][k]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int wm = (warp >> 1) * 16, wn = (warp & 1) * 32;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = tid; e < 64 * 16; e += 256) {
            const int kk = e / 64, mm = e % 64;
            const int m = m0 + mm, k = k0 + kk;
            float a = 0.f, b = 0.f;
            if (m < M && k < K) a = TA ? A[(int64_t)k * lda + m] : A[(int64_t)m * lda + k];
            const int n = n0 + mm;
            if (n < N && k < K) b = TB ? B[(int64_t)n * ldb + k] : B[(int64_t)k * ldb + n];
            As[mm][kk] = __float2bfloat16_rn(a);
            Bs[mm][kk] = __float2bfloat16_rn(b);
        }
        __syncthreads();
        uint32_t af[4];
        af[0] = ld_b32(&As[wm + g][2 * t]);
        af[1] = ld_b32(&As[wm + g + 8][2 * t]);
        af[2] = ld_b32(&As[wm + g][2 * t + 8]);
        af[3] = ld_b32(&As[wm + g + 8][2 * t + 8]);
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int nn = wn + 8 * j + g;
            mma_bf16(acc[j], af, ld_b32(&Bs[nn][2 * t]), ld_b32(&Bs[nn][2 * t + 8]));
        }
        __syncthreads();
    }
    // accumulator (j, 2h + q): row g + 8h, column 8j + 2t + q of the warp tile
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int h = 0; h < 2; h++)
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const int m = m0 + wm + g + 8 * h, n = n0 + wn + 8 * j + 2 * t + q;
                if (m < M && n < N) {
                    float* c = C + (int64_t)m * ldc + n;
                    const float v = acc[j][2 * h + q];
                    *c = ACC ? *c + v : v;
                }
            }
}

__device__ __forceinline__ float gelu_t(float x)
{
    const float c = 0.7978845608028654f;  // sqrt(2 / pi)
    return 0.5f * x * (1.f + tanhf(c * (x + 0.044715f * x * x * x)));
}

__device__ __forceinline__ float gelu_t_grad(float x)
{
    const float c = 0.7978845608028654f;
    const float t = tanhf(c * (x + 0.044715f * x * x * x));
    return 0.5f * (1.f + t) + 0.5f * x * (1.f - t * t) * c * (1.f + 3.f * 0.044715f * x * x);
}

// a (pre-activation, in place + bias) and h = GELU(a), rows of width H
__global__ void k_bias_gelu(float* __restrict__ a, const float* __restrict__ b, float* __restrict__ h, int64_t rows,
                            int H)
{
    const int64_t n = rows * H;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = a[i] + b[i % H];
        a[i] = v;
        h[i] = gelu_t(v);
    }
}

// d = d * GELU'(a)
__global__ void k_gelu_bwd(float* __restrict__ d, const float* __restrict__ a, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] *= gelu_t_grad(a[i]);
}

// y (+ b3) -> u_hat; with targets: per-sample loss 1 - (u_hat . u*)^2 into
// loss[i] and dL/dy = (I - u_hat u_hat^T)(-2 (u_hat . u*) u*) / |y| * scale
__global__ void k_mlp_out(float* __restrict__ y, const float* __restrict__ b3, const float* __restrict__ U,
                          int64_t n, float scale, float* __restrict__ u_out, float* __restrict__ dy,
                          float* __restrict__ loss)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float v[3];
        for (int c = 0; c < 3; c++) v[c] = y[i * 3 + c] + b3[c];
        const float ny = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        const float inv = ny > 0.f ? 1.f / ny : 0.f;
        const float uh[3] = {v[0] * inv, v[1] * inv, v[2] * inv};
        if (u_out)
            for (int c = 0; c < 3; c++) u_out[i * 3 + c] = uh[c];
        if (!U) continue;
        const float* us = U + i * 3;
        const float dot = uh[0] * us[0] + uh[1] * us[1] + uh[2] * us[2];
        loss[i] = 1.f - dot * dot;
        const float gu[3] = {-2.f * dot * us[0], -2.f * dot * us[1], -2.f * dot * us[2]};
        const float ug = uh[0] * gu[0] + uh[1] * gu[1] + uh[2] * gu[2];
        for (int c = 0; c < 3; c++) dy[i * 3 + c] = (gu[c] - ug * uh[c]) * inv * scale;
    }
}

// out[j] (+)= sum_i d[i][j], one thread per column (fixed order)
__global__ void k_colsum(const float* __restrict__ d, int64_t rows, int cols, float* __restrict__ out, int acc)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    float s = 0.f;
    for (int64_t i = 0; i < rows; i++) s += d[i * cols + j];
    out[j] = acc ? out[j] + s : s;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// rows idx[i] of X (K wide) and U (3 wide) into contiguous batch buffers
__global__ void k_gather_rows(const float* __restrict__ X, const float* __restrict__ U, const int64_t* __restrict__ idx,
                              int64_t n, int K, float* __restrict__ Xb, float* __restrict__ Ub)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * (K + 3); t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / (K + 3);
        const int c = (int)(t - i * (K + 3));
        const int64_t s = idx[i];
        if (c < K) Xb[i * K + c] = X[s * K + c];
        else Ub[i * 3 + (c - K)] = U[s * 3 + (c - K)];
    }
}

__global__ void k_sum_partial(const float* __restrict__ v, int64_t n, double* __restrict__ out)
{
    __shared__ double s[256];
    double a = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) a += v[i];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = s[0];
}

// the products of the forward and backward passes: FP32 (the mode the
// gradient check against the FP64 oracle holds) or BF16 tensor cores
template <bool TA, bool TB, bool ACC>
void sgemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc, cudaStream_t st,
           bool bf16 = false)
{
    dim3 grid((unsigned)ceil_div(N, 64), (unsigned)ceil_div(M, 64));
    if (bf16) k_gemm_bf16<TA, TB, ACC><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc);
    else k_sgemm<TA, TB, ACC><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc);
    TTM_LAUNCH_CHECK();
}

// Standalone BF16 inference: u_hat of n rows of X [n][K] into U [n][3].
// Each warp stages 32 rows in shared memory and runs the tensor-core MLP.
template <int KX>
__global__ void __launch_bounds__(256) k_mlp_infer(const unsigned char* __restrict__ image, const float* __restrict__ X,
                                                   int K, int64_t n, float* __restrict__ U)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned char* img = smem;
    __nv_bfloat16* sx_all = reinterpret_cast<__nv_bfloat16*>(smem + kMlpImageBytes);
    float* sy_all = reinterpret_cast<float*>(smem + kMlpImageBytes + sizeof(__nv_bfloat16) * 8 * 32 * kW1S);
    mlp_image_to_smem(image, img);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __nv_bfloat16* sx = sx_all + warp * 32 * kW1S;
    float* sy = sy_all + warp * 32 * 4;
    const float* b3 = reinterpret_cast<const float*>(img + kMlpOffB3);
    const int64_t groups = (n + 31) / 32;
    for (int64_t gi = (int64_t)blockIdx.x * 8 + warp; gi < groups; gi += (int64_t)gridDim.x * 8) {
        const int64_t row = gi * 32 + lane;
        for (int k = 0; k < KX; k++)
            sx[lane * kW1S + k] = __float2bfloat16_rn(row < n && k < K ? X[row * K + k] : 0.f);
        __syncwarp();
        mlp_warp_bf16<KX>(sx, img, sy);
        __syncwarp();
        if (row < n) {
            float y0 = sy[lane * 4] + b3[0], y1 = sy[lane * 4 + 1] + b3[1], y2 = sy[lane * 4 + 2] + b3[2];
            const float nn = sqrtf(y0 * y0 + y1 * y1 + y2 * y2);
            const float inv = nn > 0.f ? 1.f / nn : 0.f;
            U[row * 3] = y0 * inv;
            U[row * 3 + 1] = y1 * inv;
            U[row * 3 + 2] = y2 * inv;
        }
        __syncwarp();
    }
}

// Training pairs from maps: X[i] = C(v_i) / ||C(v_i)||_F (zero if the norm
// is zero), U[i] = orientation at v_i; C [K][V] (order n, graded-lex).
__global__ void k_make_pairs(const float* __restrict__ C, int n_order, int K, int64_t V,
                             const float* __restrict__ orient, const int64_t* __restrict__ idx, int64_t n,
                             float* __restrict__ X, float* __restrict__ U)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = idx[i];
        float f2 = 0.f;
        int k = 0;
        for (int a = n_order; a >= 0; a--)
            for (int b = n_order - a; b >= 0; b--, k++) {
                const int c = n_order - a - b;
                float mult = 1.f;
                for (int q = 2; q <= n_order; q++) mult *= (float)q;
                for (int q = 2; q <= a; q++) mult /= (float)q;
                for (int q = 2; q <= b; q++) mult /= (float)q;
                for (int q = 2; q <= c; q++) mult /= (float)q;
                const float x = C[(int64_t)k * V + v];
                f2 += mult * x * x;
            }
        const float inv = f2 > 0.f ? rsqrtf(f2) : 0.f;
        for (k = 0; k < K; k++) X[i * K + k] = C[(int64_t)k * V + v] * inv;
        for (int c = 0; c < 3; c++) U[i * 3 + c] = orient[(int64_t)c * V + v];
    }
}

// ---------------------------------------------------------------- host --

// counter-based SplitMix64 for the initial weights
static uint64_t splitmix(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double u01(uint64_t seed, uint64_t i) { return (splitmix(seed ^ (i * 0xD1B54A32D192ED03ull)) >> 11) * 0x1.0p-53; }

// FP32 -> BF16 with round to nearest even (finite inputs)
static uint16_t bf16_rne(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

void mlp_refresh_image(ttm_mlp* M)
{
    if (!M->image_dirty && M->image.p) return;
    const int K = M->K;
    std::vector<float> p(M->np);
    TTM_CUDA_TRY(cudaMemcpy(p.data(), M->params.p, M->np * sizeof(float), cudaMemcpyDeviceToHost));
    std::vector<unsigned char> img(kMlpImageBytes, 0);
    uint16_t* W1 = reinterpret_cast<uint16_t*>(img.data() + kMlpOffW1);
    uint16_t* W2 = reinterpret_cast<uint16_t*>(img.data() + kMlpOffW2);
    uint16_t* W3 = reinterpret_cast<uint16_t*>(img.data() + kMlpOffW3);
    float* b1 = reinterpret_cast<float*>(img.data() + kMlpOffB1);
    float* b2 = reinterpret_cast<float*>(img.data() + kMlpOffB2);
    float* b3 = reinterpret_cast<float*>(img.data() + kMlpOffB3);
    const float* pW1 = p.data();
    const float* pb1 = pW1 + (size_t)kH * K;
    const float* pW2 = pb1 + kH;
    const float* pb2 = pW2 + (size_t)kH * kH;
    const float* pW3 = pb2 + kH;
    const float* pb3 = pW3 + 3 * kH;
    for (int j = 0; j < kH; j++) {
        for (int k = 0; k < K; k++) W1[j * kW1S + k] = bf16_rne(pW1[(size_t)j * K + k]);
        for (int k = 0; k < kH; k++) W2[j * kW2S + k] = bf16_rne(pW2[(size_t)j * kH + k]);
        b1[j] = pb1[j];
        b2[j] = pb2[j];
    }
    for (int o = 0; o < 3; o++) {
        for (int k = 0; k < kH; k++) W3[o * kW2S + k] = bf16_rne(pW3[o * kH + k]);
        b3[o] = pb3[o];
    }
    if (!M->image.p) M->image.alloc(kMlpImageBytes);
    TTM_CUDA_TRY(cudaMemcpy(M->image.p, img.data(), kMlpImageBytes, cudaMemcpyHostToDevice));
    M->image_dirty = false;
}

}  // namespace ttm

namespace ttm {

static void mlp_scratch(ttm_mlp* M, int64_t rows)
{
    if (rows <= M->cap) return;
    const int K = M->K;
    M->xb.alloc(rows * K * sizeof(float));
    M->ub.alloc(rows * 3 * sizeof(float));
    M->a1.alloc(rows * kH * sizeof(float));
    M->h1.alloc(rows * kH * sizeof(float));
    M->a2.alloc(rows * kH * sizeof(float));
    M->h2.alloc(rows * kH * sizeof(float));
    M->y.alloc(rows * 3 * sizeof(float));
    M->dy.alloc(rows * 3 * sizeof(float));
    M->loss.alloc(rows * sizeof(float));
    M->part.alloc(256 * sizeof(double));
    M->cap = rows;
}

struct MlpView {
    const float *W1, *b1, *W2, *b2, *W3, *b3;
};
static MlpView view(const float* p, int K)
{
    MlpView v;
    v.W1 = p;
    v.b1 = v.W1 + (size_t)kH * K;
    v.W2 = v.b1 + kH;
    v.b2 = v.W2 + (size_t)kH * kH;
    v.W3 = v.b2 + kH;
    v.b3 = v.W3 + 3 * kH;
    return v;
}

// forward of `rows` rows already in xb (and ub if targets): fills a1..h2, y;
// u_out gets u_hat if not null; with targets fills loss and dy (scaled)
static void mlp_forward_rows(ttm_mlp* M, const float* X, const float* U, int64_t rows, float* u_out, float dscale,
                             cudaStream_t st)
{
    const int K = M->K;
    const bool bf = M->bf16;
    MlpView w = view(M->params.as<float>(), K);
    float *a1 = M->a1.as<float>(), *h1 = M->h1.as<float>(), *a2 = M->a2.as<float>(), *h2 = M->h2.as<float>();
    sgemm<false, true, false>((int)rows, kH, K, X, K, w.W1, K, a1, kH, st, bf);
    k_bias_gelu<<<1024, 256, 0, st>>>(a1, w.b1, h1, rows, kH);
    TTM_LAUNCH_CHECK();
    sgemm<false, true, false>((int)rows, kH, kH, h1, kH, w.W2, kH, a2, kH, st, bf);
    k_bias_gelu<<<1024, 256, 0, st>>>(a2, w.b2, h2, rows, kH);
    TTM_LAUNCH_CHECK();
    sgemm<false, true, false>((int)rows, 3, kH, h2, kH, w.W3, kH, M->y.as<float>(), 3, st, bf);
    k_mlp_out<<<256, 256, 0, st>>>(M->y.as<float>(), w.b3, U, rows, dscale, u_out, M->dy.as<float>(),
                                   M->loss.as<float>());
    TTM_LAUNCH_CHECK();
}

// gradient of the loss of the rows in the last forward (dy already scaled),
// into g (accumulated if acc)
static void mlp_backward_rows(ttm_mlp* M, const float* X, int64_t rows, float* g, bool acc, cudaStream_t st)
{
    const int K = M->K;
    const bool bf = M->bf16;
    MlpView w = view(M->params.as<float>(), K);
    float* gW1 = g;
    float* gb1 = gW1 + (size_t)kH * K;
    float* gW2 = gb1 + kH;
    float* gb2 = gW2 + (size_t)kH * kH;
    float* gW3 = gb2 + kH;
    float* gb3 = gW3 + 3 * kH;
    float *a1 = M->a1.as<float>(), *h1 = M->h1.as<float>(), *a2 = M->a2.as<float>(), *h2 = M->h2.as<float>();
    float* dy = M->dy.as<float>();
    const int r = (int)rows;
    // dW3 = dy^T h2, db3 = colsum dy
    if (acc) sgemm<true, false, true>(3, kH, r, dy, 3, h2, kH, gW3, kH, st, bf);
    else sgemm<true, false, false>(3, kH, r, dy, 3, h2, kH, gW3, kH, st, bf);
    k_colsum<<<1, 32, 0, st>>>(dy, rows, 3, gb3, acc);
    TTM_LAUNCH_CHECK();
    // d2 = (dy W3) * GELU'(a2), reusing h2 as storage after its last use
    float* d2 = h2;
    sgemm<false, false, false>(r, kH, 3, dy, 3, w.W3, kH, d2, kH, st, bf);
    k_gelu_bwd<<<1024, 256, 0, st>>>(d2, a2, rows * kH);
    TTM_LAUNCH_CHECK();
    if (acc) sgemm<true, false, true>(kH, kH, r, d2, kH, h1, kH, gW2, kH, st, bf);
    else sgemm<true, false, false>(kH, kH, r, d2, kH, h1, kH, gW2, kH, st, bf);
    k_colsum<<<1, kH, 0, st>>>(d2, rows, kH, gb2, acc);
    TTM_LAUNCH_CHECK();
    // d1 = (d2 W2) * GELU'(a1), into h1 after its last use
    float* d1 = h1;
    sgemm<false, false, false>(r, kH, kH, d2, kH, w.W2, kH, d1, kH, st, bf);
    k_gelu_bwd<<<1024, 256, 0, st>>>(d1, a1, rows * kH);
    TTM_LAUNCH_CHECK();
    if (acc) sgemm<true, false, true>(kH, K, r, d1, kH, X, K, gW1, K, st, bf);
    else sgemm<true, false, false>(kH, K, r, d1, kH, X, K, gW1, K, st, bf);
    k_colsum<<<1, kH, 0, st>>>(d1, rows, kH, gb1, acc);
    TTM_LAUNCH_CHECK();
}

static double sum_loss(ttm_mlp* M, int64_t rows, cudaStream_t st)
{
    k_sum_partial<<<256, 256, 0, st>>>(M->loss.as<float>(), rows, M->part.as<double>());
    TTM_LAUNCH_CHECK();
    std::vector<double> h(256);
    TTM_CUDA_TRY(cudaMemcpyAsync(h.data(), M->part.p, 256 * sizeof(double), cudaMemcpyDeviceToHost, st));
    TTM_CUDA_TRY(cudaStreamSynchronize(st));
    double s = 0.0;
    for (double x : h) s += x;
    return s;
}

}  // namespace ttm

using namespace ttm;

extern "C" int64_t ttm_mlp_num_params(int n_inputs) { return n_inputs > 0 ? mlp_num_params(n_inputs) : 0; }

extern "C" ttm_status ttm_mlp_create(ttm_ctx* ctx, int n_inputs, uint64_t seed, ttm_mlp** out)
{
    if (!ctx || !out || n_inputs <= 0 || n_inputs > 128) return TTM_E_INVALID_ARG;
    ttm_mlp* M = new ttm_mlp();
    try {
        TTM_CUDA_TRY(cudaSetDevice(ctx->device));
        M->ctx = ctx;
        M->K = n_inputs;
        M->np = mlp_num_params(n_inputs);
        M->params.alloc(M->np * sizeof(float));
        M->grad.alloc(M->np * sizeof(float));
        M->m.alloc(M->np * sizeof(float));
        M->v.alloc(M->np * sizeof(float));
        // weights ~ N(0, 1/fan_in) by Box-Muller on SplitMix64 counters, biases 0
        std::vector<float> h(M->np, 0.f);
        const int K = n_inputs;
        auto fill = [&](size_t off, int64_t count, int fan_in, uint64_t stream) {
            const double sd = 1.0 / std::sqrt((double)fan_in);
            for (int64_t i = 0; i < count; i++) {
                double u1 = u01(seed + stream, 2 * i), u2 = u01(seed + stream, 2 * i + 1);
                double z = std::sqrt(-2.0 * std::log1p(-u1)) * std::cos(2.0 * M_PI * u2);
                h[off + i] = (float)(sd * z);
            }
        };
        fill(0, (int64_t)kH * K, K, 1);
        fill((size_t)kH * K + kH, (int64_t)kH * kH, kH, 2);
        fill((size_t)kH * K + kH + kH * kH + kH, 3 * kH, kH, 3);
        TTM_CUDA_TRY(cudaMemcpy(M->params.p, h.data(), M->np * sizeof(float), cudaMemcpyHostToDevice));
        TTM_CUDA_TRY(cudaMemset(M->m.p, 0, M->np * sizeof(float)));
        TTM_CUDA_TRY(cudaMemset(M->v.p, 0, M->np * sizeof(float)));
        *out = M;
        return TTM_OK;
    } catch (const Error& e) {
        delete M;
        return (ttm_status)fail(ctx, e);
    }
}

extern "C" void ttm_mlp_destroy(ttm_mlp* mlp) { delete mlp; }

extern "C" int ttm_mlp_inputs(const ttm_mlp* mlp) { return mlp ? mlp->K : 0; }

extern "C" ttm_status ttm_mlp_get_params(const ttm_mlp* mlp, float* h_params)
{
    if (!mlp || !h_params) return TTM_E_INVALID_ARG;
    try {
        TTM_CUDA_TRY(cudaMemcpy(h_params, mlp->params.p, mlp->np * sizeof(float), cudaMemcpyDeviceToHost));
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(mlp->ctx, e);
    }
}

extern "C" ttm_status ttm_mlp_set_params(ttm_mlp* mlp, const float* h_params)
{
    if (!mlp || !h_params) return TTM_E_INVALID_ARG;
    try {
        TTM_CUDA_TRY(cudaMemcpy(mlp->params.p, h_params, mlp->np * sizeof(float), cudaMemcpyHostToDevice));
        TTM_CUDA_TRY(cudaMemset(mlp->m.p, 0, mlp->np * sizeof(float)));
        TTM_CUDA_TRY(cudaMemset(mlp->v.p, 0, mlp->np * sizeof(float)));
        mlp->step = 0;
        mlp->image_dirty = true;
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(mlp->ctx, e);
    }
}

extern "C" ttm_status ttm_mlp_forward(ttm_mlp* mlp, const float* d_X, int64_t n, float* d_U, void* stream)
{
    if (!mlp || !d_X || !d_U || n < 0) return TTM_E_INVALID_ARG;
    try {
        cudaStream_t st = (cudaStream_t)stream;
        const int64_t chunk = 65536;
        mlp_scratch(mlp, std::min<int64_t>(std::max<int64_t>(n, 1), chunk));
        for (int64_t s = 0; s < n; s += chunk) {
            const int64_t r = std::min(chunk, n - s);
            mlp_forward_rows(mlp, d_X + s * mlp->K, nullptr, r, d_U + s * 3, 1.f, st);
        }
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(mlp->ctx, e);
    }
}

extern "C" ttm_status ttm_mlp_loss_grad(ttm_mlp* mlp, const float* d_X, const float* d_U, int64_t n, float* d_grad,
                                        double* h_loss, void* stream)
{
    if (!mlp || !d_X || !d_U || !d_grad || n <= 0) return TTM_E_INVALID_ARG;
    try {
        cudaStream_t st = (cudaStream_t)stream;
        const int64_t chunk = 65536;
        mlp_scratch(mlp, std::min(n, chunk));
        double L = 0.0;
        for (int64_t s = 0; s < n; s += chunk) {
            const int64_t r = std::min(chunk, n - s);
            mlp_forward_rows(mlp, d_X + s * mlp->K, d_U + s * 3, r, nullptr, 1.f, st);
            mlp_backward_rows(mlp, d_X + s * mlp->K, r, d_grad, s > 0, st);
            L += sum_loss(mlp, r, st);
        }
        if (h_loss) *h_loss = L;
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(mlp->ctx, e);
    }
}

extern "C" ttm_status ttm_mlp_train(ttm_mlp* mlp, const float* d_X, const float* d_U, int64_t n, int epochs, int batch,
                                    float lr, uint64_t seed, double* h_last_loss, void* stream)
{
    if (!mlp || !d_X || !d_U || n <= 0 || epochs <= 0 || batch <= 0 || !(lr > 0)) return TTM_E_INVALID_ARG;
    try {
        cudaStream_t st = (cudaStream_t)stream;
        const int64_t B = std::min<int64_t>(batch, n);
        mlp_scratch(mlp, B);
        const int K = mlp->K;
        std::vector<int64_t> perm(n);
        DevBuf dperm;
        dperm.alloc(n * sizeof(int64_t));
        double last = 0.0;
        for (int ep = 0; ep < epochs; ep++) {
            // Fisher-Yates with SplitMix64 counters
            for (int64_t i = 0; i < n; i++) perm[i] = i;
            for (int64_t i = n - 1; i > 0; i--) {
                int64_t j = (int64_t)(u01(seed + 17 + ep, i) * (double)(i + 1));
                if (j > i) j = i;
                std::swap(perm[i], perm[j]);
            }
            TTM_CUDA_TRY(cudaMemcpyAsync(dperm.p, perm.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, st));
            double ep_loss = 0.0;
            for (int64_t b0 = 0; b0 + B <= n; b0 += B) {
                k_gather_rows<<<512, 256, 0, st>>>(d_X, d_U, dperm.as<int64_t>() + b0, B, K, mlp->xb.as<float>(),
                                                   mlp->ub.as<float>());
                TTM_LAUNCH_CHECK();
                // mean loss over the batch
                mlp_forward_rows(mlp, mlp->xb.as<float>(), mlp->ub.as<float>(), B, nullptr, 1.f / (float)B, st);
                mlp_backward_rows(mlp, mlp->xb.as<float>(), B, mlp->grad.as<float>(), false, st);
                mlp->step++;
                const float b1 = 0.9f, b2 = 0.999f;
                const float c1 = 1.f - std::pow(b1, (float)mlp->step), c2 = 1.f - std::pow(b2, (float)mlp->step);
                k_adam<<<512, 256, 0, st>>>(mlp->params.as<float>(), mlp->grad.as<float>(), mlp->m.as<float>(),
                                            mlp->v.as<float>(), mlp->np, lr, b1, b2, 1e-8f, c1, c2);
                TTM_LAUNCH_CHECK();
                if (b0 + 2 * B > n) ep_loss = sum_loss(mlp, B, st) / (double)B;
            }
            last = ep_loss;
        }
        TTM_CUDA_TRY(cudaStreamSynchronize(st));
        mlp->image_dirty = true;
        if (h_last_loss) *h_last_loss = last;
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(mlp->ctx, e);
    }
}

// file: "TTMMLP1\0", int32 K, int32 H, int64 nparams, float params[]
extern "C" ttm_status ttm_mlp_save(const ttm_mlp* mlp, const char* path)
{
    if (!mlp || !path) return TTM_E_INVALID_ARG;
    std::vector<float> h(mlp->np);
    ttm_status s = ttm_mlp_get_params(mlp, h.data());
    if (s != TTM_OK) return s;
    FILE* f = std::fopen(path, "wb");
    if (!f) return TTM_E_INVALID_ARG;
    const char magic[8] = {'T', 'T', 'M', 'M', 'L', 'P', '1', 0};
    int32_t K = mlp->K, H = kH;
    int64_t np = mlp->np;
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(&K, 4, 1, f) == 1 && std::fwrite(&H, 4, 1, f) == 1 &&
              std::fwrite(&np, 8, 1, f) == 1 && std::fwrite(h.data(), sizeof(float), np, f) == (size_t)np;
    std::fclose(f);
    return ok ? TTM_OK : TTM_E_INTERNAL;
}

extern "C" ttm_status ttm_mlp_load(ttm_ctx* ctx, const char* path, ttm_mlp** out)
{
    if (!ctx || !path || !out) return TTM_E_INVALID_ARG;
    FILE* f = std::fopen(path, "rb");
    if (!f) return TTM_E_INVALID_ARG;
    char magic[8];
    int32_t K = 0, H = 0;
    int64_t np = 0;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "TTMMLP1", 7) == 0 && std::fread(&K, 4, 1, f) == 1 &&
              std::fread(&H, 4, 1, f) == 1 && std::fread(&np, 8, 1, f) == 1 && H == kH && K > 0 && K <= 128 &&
              np == mlp_num_params(K);
    std::vector<float> h;
    if (ok) {
        h.resize(np);
        ok = std::fread(h.data(), sizeof(float), np, f) == (size_t)np;
    }
    std::fclose(f);
    if (!ok) return TTM_E_INVALID_ARG;
    ttm_status s = ttm_mlp_create(ctx, K, 0, out);
    if (s != TTM_OK) return s;
    return ttm_mlp_set_params(*out, h.data());
}

extern "C" ttm_status ttm_mlp_infer(ttm_mlp* mlp, const float* d_X, int64_t n, float* d_U, void* stream)
{
    if (!mlp || !d_X || !d_U || n < 0) return TTM_E_INVALID_ARG;
    try {
        TTM_CUDA_TRY(cudaSetDevice(mlp->ctx->device));
        mlp_refresh_image(mlp);
        if (n == 0) return TTM_OK;
        const size_t smem = kMlpImageBytes + sizeof(__nv_bfloat16) * 8 * 32 * kW1S + sizeof(float) * 8 * 32 * 4;
        const int64_t groups = (n + 31) / 32;
        const int grid = (int)std::min<int64_t>((groups + 7) / 8, (int64_t)mlp->ctx->num_sms * 8);
        cudaStream_t st = (cudaStream_t)stream;
        if (mlp_kx(mlp->K) == 16) {
            TTM_CUDA_TRY(cudaFuncSetAttribute(k_mlp_infer<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_mlp_infer<16><<<grid, 256, smem, st>>>(mlp->image.as<unsigned char>(), d_X, mlp->K, n, d_U);
        } else if (mlp_kx(mlp->K) == 32) {
            TTM_CUDA_TRY(cudaFuncSetAttribute(k_mlp_infer<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_mlp_infer<32><<<grid, 256, smem, st>>>(mlp->image.as<unsigned char>(), d_X, mlp->K, n, d_U);
        } else {
            throw Error{E_UNSUPPORTED, "tensor-core inference takes at most 32 inputs"};
        }
        TTM_LAUNCH_CHECK();
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(mlp->ctx, e);
    }
}

extern "C" ttm_status ttm_mlp_make_pairs(ttm_ctx* ctx, const float* d_C, int order_n, int64_t V, const float* d_orient,
                                         const int64_t* d_idx, int64_t n, float* d_X, float* d_U, void* stream)
{
    if (!ctx) return TTM_E_INVALID_ARG;
    try {
        TTM_REQUIRE(d_C && d_orient && d_idx && d_X && d_U && V > 0 && n >= 0, E_INVALID_ARG, "bad argument");
        TTM_REQUIRE(order_n >= 1 && order_n <= 12, E_UNSUPPORTED, "order out of range");
        TTM_CUDA_TRY(cudaSetDevice(ctx->device));
        if (n == 0) return TTM_OK;
        const int K = (order_n + 1) * (order_n + 2) / 2;
        k_make_pairs<<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 4096), 256, 0, (cudaStream_t)stream>>>(
            d_C, order_n, K, V, d_orient, d_idx, n, d_X, d_U);
        TTM_LAUNCH_CHECK();
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(ctx, e);
    }
}

extern "C" ttm_status ttm_mlp_set_precision(ttm_mlp* mlp, int mode)
{
    if (!mlp || (mode != TTM_MLP_FP32 && mode != TTM_MLP_BF16)) return TTM_E_INVALID_ARG;
    mlp->bf16 = mode == TTM_MLP_BF16;
    return TTM_OK;
}
