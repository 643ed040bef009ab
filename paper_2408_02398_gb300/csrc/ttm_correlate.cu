// ttm_correlate.cu -- Alg. 2 (tensorial field) on the GPU:
//   C_alpha = w * IFFT( FFT(g) * conj(FFT(T_alpha)) )       (Eqs. 5, 8)
//
// The template spectra are kept "partial": transformed along x and y only,
// on the template's own z rows (tz of the Z rows), so the plan holds
// K * tz * Y * (X/2+1) values instead of K * Z * Y * (X/2+1). The inverse
// transform of every component starts with a fused z pass: one CTA loads a
// tile of image-spectrum columns once, and for each component places the
// tz template rows on their wrapped z positions, finishes the template
// transform along z, multiplies by the image spectrum (conjugated template)
// and transforms back along z. Then a y pass over all K components and an
// x pass (complex-to-real) whose epilogue multiplies by w(x) and writes C.

#include <algorithm>
#include <vector>

#include "fft_reg.cuh"
#include "ttm_internal.h"

namespace ttm {

// component alpha of the FP64 field, placed at the origin of a tz x Y x X
// grid (wrapped in y and x; z rows are the template's rows j = 0..tz-1)
struct SrcFieldRows {
    const double* T;
    int Y, X, ty, tx;
    __device__ double operator()(int64_t row, int x) const
    {
        int j = (int)(row / Y), y = (int)(row - (int64_t)j * Y);
        int iy = wrap_to_template(y, Y, ty), ix = wrap_to_template(x, X, tx);
        if (iy < 0 || ix < 0) return 0.0;
        return T[((int64_t)j * ty + iy) * tx + ix];
    }
};

__global__ void k_spec_store(const double2* __restrict__ src, int64_t n, double scale, float2* __restrict__ dst)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 v = src[i];
        dst[i] = make_float2((float)(v.x * scale), (float)(v.y * scale));
    }
}

// Fused z pass. Columns c in [0, ncols) (ncols = Y * Xh) are the (ky, kx)
// pairs; element z of column c is at z * ncols + c. One CTA owns W adjacent
// columns. Shared memory: 3 * W * ld + Z complex.
template <typename TS, typename TW>
__global__ void __launch_bounds__(256)
k_zcorr(const float2* __restrict__ G, const TS* __restrict__ spec, int K, int tzn, int cz, int64_t ncols,
        TW* __restrict__ out, LenPlan pl, int W, int ld, const float* __restrict__ gmax, float oscale)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* gs = reinterpret_cast<float2*>(smem_raw);
    float2* bufa = gs + W * ld;
    float2* bufb = bufa + W * ld;
    float2* tws = bufb + W * ld;
    const int Z = pl.L;
    const int64_t c0 = (int64_t)blockIdx.x * W;
    load_twiddles<float>(tws, pl);
    const float gsc = (gmax && *gmax > 0.f) ? 1.f / *gmax : 1.f;
    for (int idx = threadIdx.x; idx < W * Z; idx += blockDim.x) {
        int z = idx / W, w = idx - z * W;
        int64_t c = c0 + w;
        gs[w * ld + z] = c < ncols ? cscale(G[(int64_t)z * ncols + c], gsc) : make_float2(0.f, 0.f);
    }
    const int64_t comp_stride = (int64_t)tzn * ncols;
    const int64_t out_stride = (int64_t)Z * ncols;
    for (int a = 0; a < K; a++) {
        // template rows j land on z = (j - cz) mod Z, i.e. j = (z + cz) mod Z
        const TS* sp = spec + a * comp_stride;
        for (int idx = threadIdx.x; idx < W * Z; idx += blockDim.x) {
            int z = idx / W, w = idx - z * W;
            int64_t c = c0 + w;
            int j = z + cz;
            if (j >= Z) j -= Z;
            float2 v = make_float2(0.f, 0.f);
            if (j < tzn && c < ncols) v = load_cx(sp[(int64_t)j * ncols + c]);
            bufa[w * ld + z] = v;
        }
        __syncthreads();
        float2* p = smem_fft<-1, float>(bufa, bufb, ld, W, pl, tws);
        float2* q = (p == bufa) ? bufb : bufa;
        for (int idx = threadIdx.x; idx < W * Z; idx += blockDim.x) {
            int w = idx / Z, z = idx - w * Z;
            p[w * ld + z] = cmulconj(gs[w * ld + z], p[w * ld + z]);
        }
        __syncthreads();
        float2* r = smem_fft<+1, float>(p, q, ld, W, pl, tws);
        TW* o = out + a * out_stride;
        for (int idx = threadIdx.x; idx < W * Z; idx += blockDim.x) {
            int z = idx / W, w = idx - z * W;
            int64_t c = c0 + w;
            if (c < ncols) store_cx(o + (int64_t)z * ncols + c, cscale(r[w * ld + z], oscale));
        }
        __syncthreads();
    }
}

// epilogue of the x pass: C_alpha(x) = w(x) * value
struct SinkNormalise {
    float* C;
    const float* w;
    int64_t V;
    int X;
    __device__ void operator()(int batch, int64_t row, int x, float v) const
    {
        int64_t i = row * X + x;
        // w is read-only for the whole pass: the read-only path lets these
        // loads be issued ahead of the stores to C. C is written once and
        // read back only by the maximiser: streaming (evict-first) stores
        // keep it from displacing what the passes reuse in L2.
        __stcs(C + (int64_t)batch * V + i, __ldg(w + i) * v);
    }
};

// ------------------------------------------- 16-bit spectra (FP16 / BF16)

template <typename T16>
__global__ void k_spec_store16(const double2* __restrict__ src, int64_t n, double scale, T16* __restrict__ dst)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 v = src[i];
        store_cx(dst + i, make_float2((float)(v.x * scale), (float)(v.y * scale)));
    }
}

// per-block max |v| of a double2 array (host finishes the reduction)
__global__ void k_maxabs_d2(const double2* __restrict__ v, int64_t n, double* __restrict__ part)
{
    __shared__ double s[256];
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, hypot(v[i].x, v[i].y));
    s[threadIdx.x] = m;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) s[threadIdx.x] = fmax(s[threadIdx.x], s[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// *out = max |G| (out zeroed first; non-negative floats order as their bits)
__global__ void k_maxabs_f2(const float2* __restrict__ v, int64_t n, unsigned int* __restrict__ out)
{
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, sqrtf(v[i].x * v[i].x + v[i].y * v[i].y));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// y-pass store into 16-bit pairs, times q
template <typename T16> struct StoreTo16 {
    T16* out;
    int64_t os, s;
    float q;
    __device__ __forceinline__ void operator()(float2 v, int64_t o, int64_t i, int j) const
    {
        store_cx(out + o * os + i + (int64_t)j * s, make_float2(v.x * q, v.y * q));
    }
};

// x-pass epilogue of the 16-bit path: C_alpha(x) = w(x) * value * fac[alpha]
// * max |G| (undoing the component, image-spectrum and y-pass scales)
struct SinkNormaliseScaled {
    float* C;
    const float* w;
    const float* fac;
    const float* gmax;
    int64_t V;
    int X;
    __device__ void operator()(int batch, int64_t row, int x, float v) const
    {
        int64_t i = row * X + x;
        const float g = __ldg(gmax);
        __stcs(C + (int64_t)batch * V + i, __ldg(w + i) * v * (__ldg(fac + batch) * (g > 0.f ? g : 1.f)));
    }
};

template <typename TS, typename TW>
void launch_zcorr(const float2* G, const TS* spec, int K, int tzn, int cz, int64_t ncols, TW* out,
                  const LenPlan& pz, const float* gmax, float oscale, cudaStream_t st, const DeviceWait* dw)
{
    if (dw && launch_zcorr_tma(G, spec, K, tzn, cz, ncols, out, pz, gmax, oscale, *dw, st)) return;
    if (launch_zcorr_fs(G, spec, K, tzn, cz, ncols, out, pz, gmax, oscale, st)) return;
    const int Z = pz.L;
    const int ld = (Z % 2 == 0) ? Z + 1 : Z;
    int W = (pz.tile_w >= 2 && pz.tile_w <= 16) ? pz.tile_w : 16;
    while (W > 2 && (3 * (size_t)W * ld + Z) * sizeof(float2) > 112 * 1024) W /= 2;
    size_t smem = (3 * (size_t)W * ld + Z) * sizeof(float2);
    set_smem(k_zcorr<TS, TW>, smem);
    int64_t grid = ceil_div(ncols, W);
    k_zcorr<TS, TW><<<(unsigned)grid, 256, smem, st>>>(G, spec, K, tzn, cz, ncols, out, pz, W, ld, gmax, oscale);
    TTM_LAUNCH_CHECK();
}

template void launch_zcorr<float2, float2>(const float2*, const float2*, int, int, int, int64_t, float2*,
                                           const LenPlan&, const float*, float, cudaStream_t, const DeviceWait*);
template void launch_zcorr<__half2, __half2>(const float2*, const __half2*, int, int, int, int64_t, __half2*,
                                             const LenPlan&, const float*, float, cudaStream_t, const DeviceWait*);
template void launch_zcorr<__nv_bfloat162, __nv_bfloat162>(const float2*, const __nv_bfloat162*, int, int, int,
                                                           int64_t, __nv_bfloat162*, const LenPlan&, const float*,
                                                           float, cudaStream_t, const DeviceWait*);

// FP32 partial template spectra of all K components on the grid of p
// (scaled by 1 / V of the working grid), p.zc as scratch
void spectra_fp32(Prep& p, int K, const double* d_field, float2* spec, cudaStream_t st)
{
    const int Y = p.Y, X = p.X, Xh = p.Xh, tz = p.tz, ty = p.ty, tx = p.tx;
    const int64_t V = (int64_t)p.Z * Y * X;
    const int64_t ncomp = (int64_t)tz * Y * Xh;
    double2* scratch = p.zc.as<double2>();
    for (int a = 0; a < K; a++) {
        const double* Ta = d_field + (int64_t)a * tz * ty * tx;
        launch_r2c_any<double>(SrcFieldRows{Ta, Y, X, ty, tx}, (int64_t)tz * Y, scratch, p.px64, st);
        launch_strided_any<double, -1>(scratch, StridedAxis{Xh, tz, (int64_t)Y * Xh, Xh}, p.py64,
                                   ProIdentity<double>(), StoreTo<double>{scratch, (int64_t)Y * Xh, Xh}, st);
        k_spec_store<<<1024, 256, 0, st>>>(scratch, ncomp, 1.0 / (double)V, spec + a * ncomp);
        TTM_LAUNCH_CHECK();
    }
}

// the three K-component passes of the FP32 correlate (after the per-image
// preparation of p): fused z pass, y pass, x pass with the w epilogue
void passes_fp32(Prep& p, int K, const float2* spec, float2* work, float* C, cudaStream_t st, const DeviceWait* dw)
{
    const int Z = p.Z, Y = p.Y, X = p.X, Xh = p.Xh;
    const int64_t ncols = (int64_t)Y * Xh;
    const int64_t V = (int64_t)Z * Y * X;
    launch_zcorr(p.G.as<float2>(), spec, K, p.tz, p.tz / 2, ncols, work, p.pz32, (const float*)nullptr, 1.f, st, dw);
    launch_strided_any<float, +1>(work, StridedAxis{Xh, (int64_t)K * Z, ncols, Xh}, p.py32, ProIdentity<float>(),
                                  StoreTo<float>{work, ncols, Xh}, st);
    launch_c2r_any<float>(work, (int64_t)Z * Y, SinkNormalise{C, p.w.as<float>(), V, X}, p.px32, K, st);
}

void plan_build_spectra(ttm_plan* P, const double* d_field)
{
    Prep& p = P->prep;
    const int Y = p.Y, X = p.X, Xh = p.Xh, tz = p.tz, ty = p.ty, tx = p.tx;
    const int64_t V = (int64_t)p.Z * Y * X;
    const int64_t ncomp = (int64_t)tz * Y * Xh;
    const bool half = P->prec != TTM_PREC_FP32;
    P->spec.alloc(P->K * ncomp * (half ? sizeof(__half2) : sizeof(float2)));
    double2* scratch = p.zc.as<double2>();  // tz*Y*Xh <= Z*Y*X
    cudaStream_t st = 0;
    // 16-bit spectra: the partial spectrum of component alpha is stored
    // times s_alpha = 1 / max |partial spectrum| (so |stored| <= 1) and the
    // image spectrum is used divided by max |G|. The z transform of the tz
    // template rows is then <= tz, so after the inverse z pass |v| <= Z tz
    // and after the y pass |v| <= Z tz Y (times the z-store factor): the
    // z- and y-pass stores scale by qz and q to keep these bounds under 2^15.
    const double bz = (double)p.Z * tz;
    P->work_qz = half ? (float)std::min(1.0, 32768.0 / bz) : 1.f;
    P->work_q = half ? (float)std::min(1.0, 32768.0 / (bz * P->work_qz * Y)) : 1.f;
    std::vector<float> fac(P->K, 1.f);
    DevBuf part;
    if (half) part.alloc(256 * sizeof(double));
    for (int a = 0; a < P->K; a++) {
        const double* Ta = d_field + (int64_t)a * tz * ty * tx;
        launch_r2c_any<double>(SrcFieldRows{Ta, Y, X, ty, tx}, (int64_t)tz * Y, scratch, p.px64, st);
        launch_strided_any<double, -1>(scratch, StridedAxis{Xh, tz, (int64_t)Y * Xh, Xh}, p.py64,
                                   ProIdentity<double>(), StoreTo<double>{scratch, (int64_t)Y * Xh, Xh}, st);
        if (!half) {
            k_spec_store<<<1024, 256, 0, st>>>(scratch, ncomp, 1.0 / (double)V, P->spec.as<float2>() + a * ncomp);
            TTM_LAUNCH_CHECK();
            continue;
        }
        k_maxabs_d2<<<256, 256, 0, st>>>(scratch, ncomp, part.as<double>());
        TTM_LAUNCH_CHECK();
        std::vector<double> hp(256);
        TTM_CUDA_TRY(cudaMemcpyAsync(hp.data(), part.p, 256 * sizeof(double), cudaMemcpyDeviceToHost, st));
        TTM_CUDA_TRY(cudaStreamSynchronize(st));
        double mx = 0.0;
        for (double v : hp) mx = std::max(mx, v);
        const double sa = mx > 0.0 ? 1.0 / mx : 1.0;  // on the unnormalised spectrum
        fac[a] = (float)(1.0 / (V * sa * (double)P->work_qz * (double)P->work_q));
        if (P->prec == TTM_PREC_FP16_SPECTRA)
            k_spec_store16<__half2><<<1024, 256, 0, st>>>(scratch, ncomp, sa, P->spec.as<__half2>() + a * ncomp);
        else
            k_spec_store16<__nv_bfloat162><<<1024, 256, 0, st>>>(scratch, ncomp, sa,
                                                                 P->spec.as<__nv_bfloat162>() + a * ncomp);
        TTM_LAUNCH_CHECK();
    }
    if (half) {
        P->spec_scale.alloc(P->K * sizeof(float));
        TTM_CUDA_TRY(cudaMemcpy(P->spec_scale.p, fac.data(), P->K * sizeof(float), cudaMemcpyHostToDevice));
        P->gmax.alloc(sizeof(float));
    }
    TTM_CUDA_TRY(cudaStreamSynchronize(st));
}

// z, y and x passes with 16-bit spectra and work buffer (FP32 arithmetic)
template <typename T16>
static void correlate_passes16(ttm_plan* P, float* d_C, cudaStream_t st)
{
    Prep& p = P->prep;
    const int Z = p.Z, Y = p.Y, X = p.X, Xh = p.Xh;
    const int64_t ncols = (int64_t)Y * Xh;
    const int64_t V = (int64_t)Z * Y * X;
    float* gmax = P->gmax.as<float>();
    TTM_CUDA_TRY(cudaMemsetAsync(gmax, 0, sizeof(float), st));
    k_maxabs_f2<<<(unsigned)std::min<int64_t>(ceil_div(Z * ncols, 256), (int64_t)P->ctx->num_sms * 8), 256, 0, st>>>(
        p.G.as<float2>(), Z * ncols, reinterpret_cast<unsigned int*>(gmax));
    TTM_LAUNCH_CHECK();
    T16* work = P->work.as<T16>();
    const DeviceWait dw = P->ctx->wait();
    launch_zcorr(p.G.as<float2>(), P->spec.as<T16>(), P->K, p.tz, p.tz / 2, ncols, work, p.pz32,
                 (const float*)gmax, P->work_qz, st, &dw);
    stage_end(P, ST_ZCORR, st);
    launch_strided_any<float, +1>(work, StridedAxis{Xh, (int64_t)P->K * Z, ncols, Xh}, p.py32, ProIdentity<float>(),
                                  StoreTo16<T16>{work, ncols, Xh, P->work_q}, st);
    stage_end(P, ST_YPASS, st);
    launch_c2r_any<float>(work, (int64_t)Z * Y,
                          SinkNormaliseScaled{d_C, p.w.as<float>(), P->spec_scale.as<float>(), gmax, V, X}, p.px32,
                          P->K, st);
    stage_end(P, ST_XPASS, st);
}

void correlate_run(ttm_plan* P, const float* d_tomo, float* d_C, cudaStream_t st)
{
    Prep& p = P->prep;
    const int Z = p.Z, Y = p.Y, X = p.X, Xh = p.Xh;
    const int64_t ncols = (int64_t)Y * Xh;
    const int64_t V = (int64_t)Z * Y * X;
    stage_begin(P, st);
    prep_filter(p, d_tomo, st);
    stage_end(P, ST_FILTER, st);
    // (the local sums were measured running on a second stream beside the
    // spectrum and the z/y passes: both slowed down by as much as they
    // overlapped, so they run in sequence)
    prep_localsums(p, st);
    stage_end(P, ST_LOCALSUM, st);
    prep_spectrum(p, st);
    stage_end(P, ST_SPECTRUM, st);
    if (P->prec == TTM_PREC_FP16_SPECTRA) {
        correlate_passes16<__half2>(P, d_C, st);
        return;
    }
    if (P->prec == TTM_PREC_BF16_SPECTRA) {
        correlate_passes16<__nv_bfloat162>(P, d_C, st);
        return;
    }
    float2* work = P->work.as<float2>();
    const DeviceWait dw = P->ctx->wait();
    launch_zcorr(p.G.as<float2>(), P->spec.as<float2>(), P->K, p.tz, p.tz / 2, ncols, work, p.pz32,
                 (const float*)nullptr, 1.f, st, &dw);
    stage_end(P, ST_ZCORR, st);
    launch_strided_any<float, +1>(work, StridedAxis{Xh, (int64_t)P->K * Z, ncols, Xh}, p.py32, ProIdentity<float>(),
                                  StoreTo<float>{work, ncols, Xh}, st);
    stage_end(P, ST_YPASS, st);
    launch_c2r_any<float>(work, (int64_t)Z * Y, SinkNormalise{d_C, p.w.as<float>(), V, X}, p.px32, P->K, st);
    stage_end(P, ST_XPASS, st);
}

}  // namespace ttm

using namespace ttm;

static bool params_ok(const ttm_field_params* fp, std::string& why)
{
    if (!fp) { why = "params is NULL"; return false; }
    if (fp->order_n < 2 || fp->order_n > 6 || fp->order_n % 2) { why = "order_n must be 2, 4 or 6"; return false; }
    if (fp->dprime != 3 && fp->dprime != 4) { why = "dprime must be 3 or 4"; return false; }
    if (!(fp->mask_radius > 0)) { why = "mask_radius must be positive"; return false; }
    if (!(fp->mask_soft_width >= 0)) { why = "mask_soft_width must be >= 0"; return false; }
    if (!(fp->filter_a >= 0 && fp->filter_a < 0.25)) { why = "filter_a must be in [0, 0.25)"; return false; }
    return true;
}

// the mask must be symmetric on the template grid: for an even extent the
// face at offset -t/2 has no mirror, so it must lie outside the mask
static bool mask_fits(int t, const ttm_field_params* fp)
{
    return (t % 2) ? (fp->mask_radius + fp->mask_soft_width <= (t - 1) / 2.0 + 1e-9)
                   : (fp->mask_radius + fp->mask_soft_width < t / 2.0);
}

extern "C" ttm_status ttm_plan_create(ttm_ctx* ctx, const double* d_field, int tz, int ty, int tx,
                                      const ttm_field_params* params, int Z, int Y, int X,
                                      ttm_precision precision, ttm_plan** out)
{
    return ttm_plan_create_padded(ctx, d_field, tz, ty, tx, params, Z, Y, X, Z, Y, X, precision, out);
}

extern "C" ttm_status ttm_plan_create_padded(ttm_ctx* ctx, const double* d_field, int tz, int ty, int tx,
                                             const ttm_field_params* params, int Zt, int Yt, int Xt, int Z,
                                             int Y, int X, ttm_precision precision, ttm_plan** out)
{
    if (!ctx) return TTM_E_INVALID_ARG;
    ttm_plan* P = nullptr;
    try {
        std::string why;
        TTM_REQUIRE(out && d_field, E_INVALID_ARG, "null pointer argument");
        TTM_REQUIRE(params_ok(params, why), E_INVALID_ARG, why);
        TTM_REQUIRE(precision == TTM_PREC_FP32 || precision == TTM_PREC_FP16_SPECTRA ||
                        precision == TTM_PREC_BF16_SPECTRA,
                    E_INVALID_ARG, "unknown precision");
        TTM_REQUIRE(tz > 0 && ty > 0 && tx > 0, E_SHAPE, "bad template shape");
        TTM_REQUIRE(mask_fits(tz, params) && mask_fits(ty, params) && mask_fits(tx, params), E_INVALID_ARG,
                    "mask radius (+ soft width) must fit symmetrically inside the template grid");
        TTM_CUDA_TRY(cudaSetDevice(ctx->device));
        P = new ttm_plan();
        P->ctx = ctx;
        P->fp = *params;
        P->K = ttm_num_components(params->order_n, params->dprime);
        P->prec = precision;
        prep_create(ctx, P->prep, Zt, Yt, Xt, Z, Y, X, tz, ty, tx, *params);

        plan_build_spectra(P, d_field);
        const int64_t Vh = (int64_t)Z * Y * P->prep.Xh;
        const size_t elem = precision == TTM_PREC_FP32 ? sizeof(float2) : sizeof(__half2);
        P->work.alloc(P->K * Vh * elem);
        const int64_t V = (int64_t)Z * Y * X;
        P->cand_cap = V / 8 + 64;  // strict 26-neighbour maxima are >= 2 apart per axis
        P->cand.alloc(P->cand_cap * (sizeof(int64_t) + sizeof(float)));
        P->cand_count.alloc(sizeof(unsigned long long));
        P->fb_count.alloc(sizeof(unsigned long long));
        TTM_CUDA_TRY(cudaMemset(P->fb_count.p, 0, sizeof(unsigned long long)));
        *out = P;
        return TTM_OK;
    } catch (const Error& e) {
        delete P;
        return (ttm_status)fail(ctx, e);
    }
}

extern "C" void ttm_plan_destroy(ttm_plan* plan) { delete plan; }

extern "C" int ttm_plan_components(const ttm_plan* plan) { return plan ? plan->K : 0; }

extern "C" void ttm_plan_valid_box(const ttm_plan* plan, int* b)
{
    if (!plan || !b) return;
    const Prep& p = plan->prep;
    b[0] = p.tz / 2; b[1] = p.Zt - (p.tz - p.tz / 2) + 1;
    b[2] = p.ty / 2; b[3] = p.Yt - (p.ty - p.ty / 2) + 1;
    b[4] = p.tx / 2; b[5] = p.Xt - (p.tx - p.tx / 2) + 1;
}

extern "C" ttm_status ttm_correlate(ttm_plan* plan, const float* d_tomo, float* d_C, void* stream)
{
    if (!plan) return TTM_E_INVALID_ARG;
    try {
        TTM_REQUIRE(d_tomo && d_C, E_INVALID_ARG, "null pointer argument");
        TTM_CUDA_TRY(cudaSetDevice(plan->ctx->device));
        correlate_run(plan, d_tomo, d_C, (cudaStream_t)stream);
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(plan->ctx, e);
    }
}

extern "C" ttm_status ttm_plan_copy_w(ttm_plan* plan, float* d_w, void* stream)
{
    if (!plan) return TTM_E_INVALID_ARG;
    try {
        TTM_REQUIRE(d_w, E_INVALID_ARG, "null pointer argument");
        const Prep& p = plan->prep;
        TTM_CUDA_TRY(cudaMemcpyAsync(d_w, p.w.p, (size_t)p.Z * p.Y * p.X * sizeof(float),
                                     cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(plan->ctx, e);
    }
}

extern "C" ttm_status ttm_plan_set_localsum(ttm_plan* plan, int mode)
{
    if (!plan || (mode != TTM_LOCALSUM_FP64 && mode != TTM_LOCALSUM_DF64)) return TTM_E_INVALID_ARG;
    plan->prep.localsum_mode = mode;
    return TTM_OK;
}
