// ttm_zcorr_tma.cu -- the fused z pass of the tensorial correlation (Alg. 2,
// Eq. 5) with its inputs staged by the Tensor Memory Accelerator.
//
// Same arithmetic as the register four-step z pass (k_fs_zcorr): per tile
// of W adjacent (ky, kx) columns, for every component the template's tz
// partial-spectrum rows are placed on their wrapped z rows, transformed
// along z, multiplied by the conjugated image spectrum in the (k1 + E k2)
// order and transformed back. The difference is how the inputs arrive:
//  * the image-spectrum tile [Z][W] is one 2-D TMA box, loaded once;
//  * the template rows of component a + 1 ([tz][W], one box) are loaded by
//    TMA into the other half of a double buffer while component a is being
//    transformed, so the per-component loads no longer stall the warps
//    (the long-scoreboard stall of the plain-load version).
// W is even, so every box starts on a 16-byte boundary (x = 2 c0 floats).
// Every wait on a copy is bounded (the context's wait limit); when one
// expires the kernel records it in the context's error word, waits (with a
// generous fixed limit) for the copies it has in flight and returns without
// writing; the host reads the record with ttm_ctx_device_status.
#include <mutex>

#include "fft_reg.cuh"
#include "tma.cuh"
#include "ttm_internal.h"

namespace ttm {

template <int E, int P> struct ZtShape {
    static constexpr int L = E * P;
    static constexpr int W = (256 / P) & ~1;  // even: 16-byte aligned boxes
    static constexpr int THREADS = W * P;
    static constexpr int KS = P + 1;
    static constexpr int LD = (E * KS) | 1;
};

__host__ __device__ constexpr size_t zt_align(size_t b, size_t a) { return (b + a - 1) / a * a; }

// shared-memory layout (bytes): image tile, two template-row buffers (each
// 128-byte aligned, the TMA destinations), twiddles, transpose, barriers
struct ZtLayout {
    size_t g, s0, s1, tw, xa, bar, total;
    __host__ __device__ ZtLayout(int Z, int W, int LD, int tzn)
    {
        g = 0;
        s0 = zt_align((size_t)Z * W * sizeof(float2), 128);
        const size_t sb = zt_align((size_t)tzn * W * sizeof(float2), 128);
        s1 = s0 + sb;
        tw = s1 + sb;
        xa = tw + zt_align((size_t)Z * sizeof(float2), 16);
        bar = xa + zt_align((size_t)W * LD * sizeof(float2), 16);
        total = bar + 3 * sizeof(uint64_t);
    }
};

constexpr long long kDrainPolls = 1ll << 22;

template <int E, int P>
__global__ void __launch_bounds__(256, 2)
k_zcorr_tma(const __grid_constant__ CUtensorMap tmG, const __grid_constant__ CUtensorMap tmS, int K, int tzn, int cz,
            int64_t ncols, float2* __restrict__ out, const void* twg, long long wait_limit, int* __restrict__ err)
{
    using S = ZtShape<E, P>;
    constexpr int Z = S::L;
    constexpr int W = S::W;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const ZtLayout lay(Z, W, S::LD, tzn);
    float2* gt = reinterpret_cast<float2*>(smem_raw + lay.g);
    float2* sbuf[2] = {reinterpret_cast<float2*>(smem_raw + lay.s0), reinterpret_cast<float2*>(smem_raw + lay.s1)};
    float2* tw = reinterpret_cast<float2*>(smem_raw + lay.tw);
    float2* xa = reinterpret_cast<float2*>(smem_raw + lay.xa);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + lay.bar);  // [0] image tile, [1], [2] template rows
    const int t = threadIdx.x;
    const int w = t % W, p = t / W;
    const int64_t c0 = (int64_t)blockIdx.x * W;
    const int64_t c = c0 + w;
    const bool act = c < ncols;
    const uint32_t sbytes = (uint32_t)(tzn * W * sizeof(float2));
    if (t == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (t == 0) {
        mbar_expect_tx(&bars[0], (uint32_t)(Z * W * sizeof(float2)));
        tma_load_2d(gt, &tmG, (int)(2 * c0), 0, &bars[0]);
        mbar_expect_tx(&bars[1], sbytes);
        tma_load_2d(sbuf[0], &tmS, (int)(2 * c0), 0, &bars[1]);
    }
    fs_load_tw<float>(tw, twg, Z);
    // a wait that expired: record it, let the copies in flight land (each
    // barrier phase waited on below has had its load issued), leave.
    // Before the loop those are the image tile and component 0; in
    // iteration a, components a and a + 1.
    if (__syncthreads_or(!mbar_wait(&bars[0], 0, wait_limit))) {
        if (t == 0) atomicExch(err, 1);
        mbar_wait(&bars[0], 0, kDrainPolls);
        mbar_wait(&bars[1], 0, kDrainPolls);
        return;
    }
    float2* xl = xa + w * S::LD;
    const float2* gl = gt + w;  // element z of this column at gl[z * W]
    for (int a = 0; a < K; a++) {
        const int buf = a & 1;
        if (t == 0 && a + 1 < K) {
            // the other buffer held component a - 1, read before the last barrier
            mbar_expect_tx(&bars[1 + (buf ^ 1)], sbytes);
            tma_load_2d(sbuf[buf ^ 1], &tmS, (int)(2 * c0), (a + 1) * tzn, &bars[1 + (buf ^ 1)]);
        }
        if (__syncthreads_or(!mbar_wait(&bars[1 + buf], (a >> 1) & 1, wait_limit))) {
            if (t == 0) atomicExch(err, 1);
            mbar_wait(&bars[1 + buf], (a >> 1) & 1, kDrainPolls);
            if (a + 1 < K) mbar_wait(&bars[1 + (buf ^ 1)], ((a + 1) >> 1) & 1, kDrainPolls);
            return;
        }
        const float2* sp = sbuf[buf] + w;
        float2 x[E];
#pragma unroll
        for (int m = 0; m < E; m++) {
            // template row j lands on z = (j - cz) mod Z
            int j = p + P * m + cz;
            if (j >= Z) j -= Z;
            x[m] = j < tzn ? sp[j * W] : make_float2(0.f, 0.f);
        }
        fs_phase1<float, E, P, -1>(x, p, xl, tw);
        __syncthreads();
#pragma unroll
        for (int ii = 0; ii < E / P; ii++)
#pragma unroll
            for (int q = 0; q < P; q++) x[ii * P + q] = xl[(p + P * ii) * S::KS + q];
        __syncthreads();
#pragma unroll
        for (int ii = 0; ii < E / P; ii++) {
            const int k1 = p + P * ii;
            float2* u = x + ii * P;
            dft_reg<P, -1, S::L, float>(u, tw);
#pragma unroll
            for (int k2 = 0; k2 < P; k2++) u[k2] = cmulconj(gl[(k1 + E * k2) * W], u[k2]);
            // inverse, backwards: P-point DFT over k2, conjugate twiddles
            dft_reg<P, +1, S::L, float>(u, tw);
#pragma unroll
            for (int q = 0; q < P; q++) {
                float2 v = u[q];
                if (q * k1 != 0) v = cmul(v, twid<+1, float>(tw, q * k1));
                xl[k1 * S::KS + q] = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k1 = 0; k1 < E; k1++) x[k1] = xl[k1 * S::KS + p];
        dft_reg<E, +1, S::L, float>(x, tw);
        if (act) {
            float2* o = out + (int64_t)a * Z * ncols + c;
#pragma unroll
            for (int m = 0; m < E; m++) o[(int64_t)(p + P * m) * ncols] = x[m];
        }
        __syncthreads();  // all reads of xl and of this buffer done
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            (void)cudaGetLastError();
    });
    return fn;
}

// 2-D FP32 view [rows][2 * ncols] of a complex array, box [box_rows][2 W]
static bool make_map(CUtensorMap& m, const float2* base, int64_t ncols, int64_t rows, int W, int box_rows)
{
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * ncols), (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(2 * ncols * sizeof(float))};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * W), (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool launch_zcorr_tma(const float2* G, const float2* spec, int K, int tzn, int cz, int64_t ncols, float2* out,
                      const LenPlan& pz, const DeviceWait& dw, cudaStream_t st)
{
    int E, P;
    const int Z = pz.L;
    if (pz.no_reg || !fs_split(Z, E, P) || Z > 256 || tzn < 1 || tzn > 256 || (ncols & 1) || !dw.err) return false;
    if ((reinterpret_cast<uintptr_t>(G) | reinterpret_cast<uintptr_t>(spec)) & 15) return false;
    bool launched = false;
#define TTM_ZT(E_, P_)                                                                                         \
    {                                                                                                          \
        using S = ZtShape<E_, P_>;                                                                             \
        CUtensorMap mg, ms;                                                                                    \
        if (!make_map(mg, G, ncols, Z, S::W, Z) || !make_map(ms, spec, ncols, (int64_t)K * tzn, S::W, tzn))    \
            break;                                                                                             \
        const size_t smem = ZtLayout(Z, S::W, S::LD, tzn).total;                                               \
        if (smem > 110 * 1024) break;                                                                          \
        auto k = k_zcorr_tma<E_, P_>;                                                                          \
        set_smem(k, smem);                                                                                     \
        k<<<(unsigned)ceil_div(ncols, S::W), S::THREADS, smem, st>>>(mg, ms, K, tzn, cz, ncols, out, pz.tw,  \
                                                                       dw.limit, dw.err);                      \
        launched = true;                                                                                       \
    }
    switch (Z) {
        case 64: TTM_ZT(8, 8); break;
        case 128: TTM_ZT(16, 8); break;
        case 200: TTM_ZT(20, 10); break;
        case 256: TTM_ZT(16, 16); break;
        default: break;
    }
#undef TTM_ZT
    if (launched) TTM_LAUNCH_CHECK();
    return launched;
}

}  // namespace ttm
