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
// W is a multiple of 4, so every box starts on a 16-byte boundary (x = c0
// complex values of 8 bytes, or of 4 bytes for 16-bit spectra).
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
    static constexpr int W = (256 / P) & ~3;  // a multiple of 4: 16-byte aligned boxes
    static constexpr int THREADS = W * P;
    static constexpr int KS = P + 1;
    static constexpr int LD = (E * KS) | 1;
};

__host__ __device__ constexpr size_t zt_align(size_t b, size_t a) { return (b + a - 1) / a * a; }

// shared-memory layout (bytes): image tile, two template-row buffers (each
// 128-byte aligned, the TMA destinations; es = bytes per stored complex
// value), twiddles, transpose, barriers
struct ZtLayout {
    size_t g, s0, s1, tw, xa, bar, total;
    __host__ __device__ ZtLayout(int Z, int W, int LD, int tzn, int es)
    {
        g = 0;
        s0 = zt_align((size_t)Z * W * sizeof(float2), 128);
        const size_t sb = zt_align((size_t)tzn * W * es, 128);
        s1 = s0 + sb;
        tw = s1 + sb;
        xa = tw + zt_align((size_t)Z * sizeof(float2), 16);
        bar = xa + zt_align((size_t)W * LD * sizeof(float2), 16);
        total = bar + 3 * sizeof(uint64_t);
    }
};

constexpr long long kDrainPolls = 1ll << 22;

// TS / TW: storage of the template spectra and of the output (float2, or
// FP16 / BF16 pairs with the image spectrum scaled by 1 / *gmax as it is
// used and the output scaled by oscale, as in the plain-load kernel)
template <int E, int P, typename TS, typename TW>
__global__ void __launch_bounds__(256, 2)
k_zcorr_tma(const __grid_constant__ CUtensorMap tmG, const __grid_constant__ CUtensorMap tmS, int K, int tzn, int cz,
            int64_t ncols, TW* __restrict__ out, const void* twg, const float* __restrict__ gmax, float oscale,
            long long wait_limit, int* __restrict__ err)
{
    using S = ZtShape<E, P>;
    constexpr int Z = S::L;
    constexpr int W = S::W;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const ZtLayout lay(Z, W, S::LD, tzn, (int)sizeof(TS));
    float2* gt = reinterpret_cast<float2*>(smem_raw + lay.g);
    TS* sbuf[2] = {reinterpret_cast<TS*>(smem_raw + lay.s0), reinterpret_cast<TS*>(smem_raw + lay.s1)};
    const float gsc = (gmax && *gmax > 0.f) ? 1.f / *gmax : 1.f;
    float2* tw = reinterpret_cast<float2*>(smem_raw + lay.tw);
    float2* xa = reinterpret_cast<float2*>(smem_raw + lay.xa);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + lay.bar);  // [0] image tile, [1], [2] template rows
    const int t = threadIdx.x;
    const int w = t % W, p = t / W;
    const int64_t c0 = (int64_t)blockIdx.x * W;
    const int64_t c = c0 + w;
    const bool act = c < ncols;
    const uint32_t sbytes = (uint32_t)(tzn * W * sizeof(TS));
    // box x coordinates in 32-bit elements: two per FP32 complex value, one
    // per 16-bit pair
    const int xg = (int)(2 * c0);
    const int xs = (int)(c0 * (int64_t)(sizeof(TS) / 4));
    if (t == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (t == 0) {
        mbar_expect_tx(&bars[0], (uint32_t)(Z * W * sizeof(float2)));
        tma_load_2d(gt, &tmG, xg, 0, &bars[0]);
        mbar_expect_tx(&bars[1], sbytes);
        tma_load_2d(sbuf[0], &tmS, xs, 0, &bars[1]);
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
            tma_load_2d(sbuf[buf ^ 1], &tmS, xs, (a + 1) * tzn, &bars[1 + (buf ^ 1)]);
        }
        if (__syncthreads_or(!mbar_wait(&bars[1 + buf], (a >> 1) & 1, wait_limit))) {
            if (t == 0) atomicExch(err, 1);
            mbar_wait(&bars[1 + buf], (a >> 1) & 1, kDrainPolls);
            if (a + 1 < K) mbar_wait(&bars[1 + (buf ^ 1)], ((a + 1) >> 1) & 1, kDrainPolls);
            return;
        }
        const TS* sp = sbuf[buf] + w;
        float2 x[E];
#pragma unroll
        for (int m = 0; m < E; m++) {
            // template row j lands on z = (j - cz) mod Z
            int j = p + P * m + cz;
            if (j >= Z) j -= Z;
            x[m] = j < tzn ? load_cx(sp[j * W]) : make_float2(0.f, 0.f);
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
            for (int k2 = 0; k2 < P; k2++) u[k2] = cmulconj(cscale(gl[(k1 + E * k2) * W], gsc), u[k2]);
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
            TW* o = out + (int64_t)a * Z * ncols + c;
#pragma unroll
            for (int m = 0; m < E; m++) store_cx(o + (int64_t)(p + P * m) * ncols, cscale(x[m], oscale));
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

// 2-D view [rows][ncols * es / 4] (32-bit elements) of an array of complex
// values of es bytes (8: FP32 pairs as two FP32 elements; 4: a 16-bit pair
// as one 32-bit element), box [box_rows][W complex values]
static bool make_map(CUtensorMap& m, const void* base, int es, int64_t ncols, int64_t rows, int W, int box_rows)
{
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const int per = es / 4;  // 32-bit elements per complex value
    const cuuint64_t dims[2] = {(cuuint64_t)(per * ncols), (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(ncols * es)};
    const cuuint32_t box[2] = {(cuuint32_t)(per * W), (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(&m, per == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 2,
               const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename TS, typename TW>
bool launch_zcorr_tma(const float2* G, const TS* spec, int K, int tzn, int cz, int64_t ncols, TW* out,
                      const LenPlan& pz, const float* gmax, float oscale, const DeviceWait& dw, cudaStream_t st)
{
    int E, P;
    const int Z = pz.L;
    constexpr int es = (int)sizeof(TS);
    // row strides of both maps a multiple of 16 bytes
    if (pz.no_reg || !fs_split(Z, E, P) || Z > 256 || tzn < 1 || tzn > 256 || (ncols * es) % 16 || (ncols & 1) ||
        !dw.err)
        return false;
    if ((reinterpret_cast<uintptr_t>(G) | reinterpret_cast<uintptr_t>(spec)) & 15) return false;
    bool launched = false;
    // box x = c0 complex values: c0 * es bytes a multiple of 16 (c0 = block * W)
#define TTM_ZT(E_, P_)                                                                                         \
    {                                                                                                          \
        using S = ZtShape<E_, P_>;                                                                             \
        static_assert(S::W % 4 == 0, "tile width keeps 4-byte boxes on 16-byte boundaries");                 \
        CUtensorMap mg, ms;                                                                                    \
        if (!make_map(mg, G, 8, ncols, Z, S::W, Z) || !make_map(ms, spec, es, ncols, (int64_t)K * tzn, S::W, tzn)) \
            break;                                                                                             \
        const size_t smem = ZtLayout(Z, S::W, S::LD, tzn, es).total;                                           \
        if (smem > 110 * 1024) break;                                                                          \
        auto k = k_zcorr_tma<E_, P_, TS, TW>;                                                                  \
        set_smem(k, smem);                                                                                     \
        k<<<(unsigned)ceil_div(ncols, S::W), S::THREADS, smem, st>>>(mg, ms, K, tzn, cz, ncols, out, pz.tw,  \
                                                                       gmax, oscale, dw.limit, dw.err);        \
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

template bool launch_zcorr_tma<float2, float2>(const float2*, const float2*, int, int, int, int64_t, float2*,
                                               const LenPlan&, const float*, float, const DeviceWait&, cudaStream_t);
template bool launch_zcorr_tma<__half2, __half2>(const float2*, const __half2*, int, int, int, int64_t, __half2*,
                                                 const LenPlan&, const float*, float, const DeviceWait&,
                                                 cudaStream_t);
template bool launch_zcorr_tma<__nv_bfloat162, __nv_bfloat162>(const float2*, const __nv_bfloat162*, int, int, int,
                                                               int64_t, __nv_bfloat162*, const LenPlan&,
                                                               const float*, float, const DeviceWait&, cudaStream_t);

}  // namespace ttm
