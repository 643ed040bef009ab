// ttm_prep.cu -- per-tomogram preparation shared by TTM and TM:
//   g = h * f (Eq. 3: separable taps [a, 1-2a, a], zero padded), FP32,
//   G = FFT(g) in FP32 (the image spectrum of Alg. 2),
//   S1 = m * g and S2 = m^2 * g^2 (Eq. 2) by one packed FP64 complex FFT of
//   g + i g^2 against the real, even spectrum of the mask, and
//   w = 1 / sqrt(S2 - S1^2 / M) (0 where the local variance is below
//   1e-8 M mean(g^2), a window too empty for the FP32 correlation to
//   resolve, or below 1e-10 S2, constant to rounding).
#include <cmath>
#include <vector>

#include "fft_reg.cuh"
#include "ttm_internal.h"

namespace ttm {

void DevBuf::alloc(size_t n)
{
    release();
    if (n == 0) return;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
        p = nullptr;
        (void)cudaGetLastError();
        throw Error{E_OOM, "cudaMalloc(" + std::to_string(n) + " bytes) failed: " + cudaGetErrorString(e)};
    }
    bytes = n;
}

void DevBuf::release()
{
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

double make_mask(int tz, int ty, int tx, double r, double soft, std::vector<double>& m)
{
    m.assign((size_t)tz * ty * tx, 0.0);
    const int cz = tz / 2, cy = ty / 2, cx = tx / 2;
    double M = 0;
    for (int z = 0; z < tz; z++)
        for (int y = 0; y < ty; y++)
            for (int x = 0; x < tx; x++) {
                double d = std::sqrt((double)(x - cx) * (x - cx) + (double)(y - cy) * (y - cy) +
                                     (double)(z - cz) * (z - cz));
                double v = 0.0;
                if (d <= r) v = 1.0;
                else if (soft > 0 && d < r + soft) v = 0.5 * (1.0 + std::cos(M_PI * (d - r) / soft));
                m[((size_t)z * ty + y) * tx + x] = v;
                M += v;
            }
    return M;
}

// ------------------------------------------------------------- kernels --

constexpr int kPreThreads = 256;

// g = h * f, the 27-point product filter (taps a, 1 - 2a, a on each axis) in
// FP32 (the input is FP32), applied separably while marching along z: a
// thread owns four consecutive voxels of one row (y, x0 .. x0+3) over a
// chunk of kPfZChunk planes. For each plane it filters the rows y-1, y, y+1
// along x (one read of x0-1 .. x0+4 each) and combines them along y; three
// such planes in registers give g along z. Writes g (f32) and (g, g^2) in
// FP64 or as double-float pairs for the local sums (unless the first
// local-sum pass forms them itself), and per-block partial sums of g^2 for
// the variance floor (fixed order).
// The tomogram f is Zt x Yt x Xt; g lives on the working grid Z x Y x X
// (>= the tomogram on every axis, zero beyond it apart from the filter's
// one-voxel spill). Only tomogram voxels enter the g^2 partial sums.
constexpr int kPreVox = 4;
constexpr int kPfZChunk = 25;

static int64_t prefilter_blocks(int Z, int Y, int X)
{
    return ceil_div((int64_t)ceil_div(Z, kPfZChunk) * Y * ceil_div(X, kPreVox), kPreThreads);
}

// DF: the (g, g^2) pack of the local sums in double-float, else in FP64;
// zc == nullptr: no pack (the first local-sum pass forms it from g32)
template <bool DF>
__global__ void __launch_bounds__(kPreThreads)
k_prefilter(const float* __restrict__ f, int Zt, int Yt, int Xt, int Z, int Y, int X, float a,
            float* __restrict__ g32, double2* __restrict__ zc, double* __restrict__ partials)
{
    __shared__ float warp_sums[kPreThreads / 32];
    const int Xq = (X + kPreVox - 1) / kPreVox;
    const int nzc = (Z + kPfZChunk - 1) / kPfZChunk;
    const int64_t nq = (int64_t)nzc * Y * Xq;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float sq = 0.f;
    if (q < nq) {
        const int xq = (int)(q % Xq);
        const int64_t r = q / Xq;
        const int y = (int)(r % Y);
        const int cz = (int)(r / Y);
        const int x0 = xq * kPreVox;
        const int z0 = cz * kPfZChunk, z1 = min(Z, z0 + kPfZChunk);
        const float t0 = a, t1 = 1.f - 2.f * a;
        // the x- and y-filtered plane zz at (y, x0 .. x0+3); zero off the tomogram
        auto plane = [&](int zz, float* o) {
#pragma unroll
            for (int k = 0; k < kPreVox; k++) o[k] = 0.f;
            if (zz < 0 || zz >= Zt) return;
#pragma unroll
            for (int dy = -1; dy <= 1; dy++) {
                const int yy = y + dy;
                if (yy < 0 || yy >= Yt) continue;
                const float* row = f + ((int64_t)zz * Yt + yy) * Xt;
                float v[kPreVox + 2];
#pragma unroll
                for (int k = 0; k < kPreVox + 2; k++) {
                    const int xx = x0 - 1 + k;
                    v[k] = (xx >= 0 && xx < Xt) ? __ldg(row + xx) : 0.f;
                }
                const float wy = dy == 0 ? t1 : t0;
#pragma unroll
                for (int k = 0; k < kPreVox; k++) o[k] += wy * (t1 * v[k + 1] + t0 * (v[k] + v[k + 2]));
            }
        };
        float pm[kPreVox], pc[kPreVox], pn[kPreVox];
        plane(z0 - 1, pm);
        plane(z0, pc);
        const bool inrow = y < Yt;
#pragma unroll 1
        for (int z = z0; z < z1; z++) {
            plane(z + 1, pn);
            const int64_t v0 = ((int64_t)z * Y + y) * X + x0;
#pragma unroll
            for (int k = 0; k < kPreVox; k++) {
                const float g = t1 * pc[k] + t0 * (pm[k] + pn[k]);
                if (x0 + k < X) {
                    g32[v0 + k] = g;
                    if (!zc) {
                    } else if (DF) {
                        // (g, g^2) as double-float pairs; g^2 is exact as hi + lo
                        const df64 s2 = two_prod(g, g);
                        reinterpret_cast<float4*>(zc)[v0 + k] = make_float4(g, 0.f, s2.hi, s2.lo);
                    } else {
                        const double gd = (double)g;
                        zc[v0 + k] = make_double2(gd, gd * gd);
                    }
                    if (inrow && z < Zt && x0 + k < Xt) sq += g * g;
                }
                pm[k] = pc[k];
                pc[k] = pn[k];
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int i = 0; i < kPreThreads / 32; i++) b += warp_sums[i];
        partials[blockIdx.x] = b;
    }
}

// floor = 1e-8 * M * mean(g^2) (fixed summation order)
__global__ void __launch_bounds__(1024)
k_var_floor(const double* __restrict__ partials, int64_t nblk, int64_t V, double M, double* floor_out)
{
    __shared__ double s2[1024];
    double b = 0;
    for (int64_t i = threadIdx.x; i < nblk; i += blockDim.x) b += partials[i];
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) s2[threadIdx.x] += s2[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) floor_out[0] = 1e-8 * M * (s2[0] / (double)V);
}

// mask placed at the origin of the Z x Y x X grid (wrapped), as real rows
struct SrcWrappedMask {
    const double* m;
    int Y, X, Z, tz, ty, tx;
    __device__ double operator()(int64_t row, int x) const
    {
        int z = (int)(row / Y), y = (int)(row - (int64_t)z * Y);
        int iz = wrap_to_template(z, Z, tz), iy = wrap_to_template(y, Y, ty), ix = wrap_to_template(x, X, tx);
        if (iz < 0 || iy < 0 || ix < 0) return 0.0;
        return m[((int64_t)iz * ty + iy) * tx + ix];
    }
};

struct SrcFloat {
    const float* g;
    int X;
    __device__ float operator()(int64_t row, int x) const { return g[row * X + x]; }
};

// real part / V of the (Hermitian half) mask spectrum on the octant
// kz <= Z/2, ky <= Y/2, kx <= X/2 (the spectrum of a mask that is symmetric
// in every axis is real and even in every axis)
__global__ void k_mhat_octant(const double2* __restrict__ spec, int Z, int Y, int Xh, int X,
                              double inv_V, double* __restrict__ oct)
{
    const int Zo = Z / 2 + 1, Yo = Y / 2 + 1, Xo = X / 2 + 1;
    int64_t n = (int64_t)Zo * Yo * Xo;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int kx = (int)(i % Xo);
        int64_t t = i / Xo;
        int ky = (int)(t % Yo), kz = (int)(t / Yo);
        oct[i] = spec[((int64_t)kz * Y + ky) * Xh + kx].x * inv_V;
    }
}

// prologue of the inverse z pass: multiply by the mask spectrum
struct ProMaskSpectrum {
    const double* oct;
    int Z, Y, X;
    __device__ double2 operator()(double2 v, int64_t, int64_t i, int kz) const
    {
        int ky = (int)(i / X), kx = (int)(i - (int64_t)ky * X);
        int az = kz <= Z - kz ? kz : Z - kz;
        int ay = ky <= Y - ky ? ky : Y - ky;
        int ax = kx <= X - kx ? kx : X - kx;
        double m = oct[((int64_t)az * (Y / 2 + 1) + ay) * (X / 2 + 1) + ax];
        return make_double2(v.x * m, v.y * m);
    }
};

// epilogue of the inverse x pass: (S1, S2) -> w
struct StoreW {
    float* w;
    const double* floor;
    double M;
    int X;
    __device__ void operator()(double2 v, int64_t l, int64_t, int j) const
    {
        double S1 = v.x, S2 = v.y;
        double var = S2 - S1 * S1 / M;
        // zero local variance: below the volume-energy floor, or constant to
        // ~5 digits over the window (the FFT leaves rounding noise there)
        w[l * X + j] = (var > floor[0] && var > 1e-10 * S2) ? (float)(1.0 / sqrt(var)) : 0.0f;
    }
};

// the (g, g^2) line of the double-float local sums formed from g as it is
// loaded: g exact in the head, g^2 exact as a TwoProd pair
struct SrcGSquared {
    const float* g;
    int X;
    __device__ dcx operator()(int64_t l, int j) const
    {
        const float v = __ldg(g + l * X + j);
        dcx r;
        r.x = df64(v, 0.f);
        r.y = two_prod(v, v);
        return r;
    }
};

// whether the first double-float local-sum pass reads g itself (a length
// with the three-level register kernel), so the prefilter writes no pack
static bool localsum_reads_g(const Prep& p) { return p.localsum_mode == 1 && !p.pxd.no_reg && line3_length(p.X); }

// double-float versions of the mask-spectrum prologue and the w epilogue
struct ProMaskSpectrumDF {
    const float2* oct;
    int Z, Y, X;
    __device__ dcx operator()(dcx v, int64_t, int64_t i, int kz) const
    {
        int ky = (int)(i / X), kx = (int)(i - (int64_t)ky * X);
        int az = kz <= Z - kz ? kz : Z - kz;
        int ay = ky <= Y - ky ? ky : Y - ky;
        int ax = kx <= X - kx ? kx : X - kx;
        const float2 m2 = oct[((int64_t)az * (Y / 2 + 1) + ay) * (X / 2 + 1) + ax];
        const df64 m(m2.x, m2.y);
        dcx o;
        o.x = v.x * m;
        o.y = v.y * m;
        return o;
    }
};

struct StoreWDF {
    float* w;
    const double* floor;
    df64 inv_M;
    int X;
    __device__ void operator()(dcx v, int64_t l, int64_t, int j) const
    {
        const df64 S1 = v.x, S2 = v.y;
        const df64 var = S2 - (S1 * S1) * inv_M;  // the cancellation happens here, in double-float
        const float vf = var.hi + var.lo;
        const bool pos = vf > (float)floor[0] && vf > 1e-10f * (S2.hi + S2.lo);
        w[l * X + j] = pos ? rsqrtf(vf) : 0.0f;
    }
};

// Fused z pass of the local sums: per tile of W adjacent (y, x) columns,
// the forward transform along z, the product with the (real, even) mask
// spectrum and the inverse transform, through shared memory (Stockham
// stages: one copy of each butterfly, which keeps the long FP64 /
// double-float kernels inside the instruction cache). One read and one
// write of the (g, g^2) spectrum instead of two each.
template <typename R, class Mask>
__global__ void __launch_bounds__(256)
k_zmask(cx<R>* __restrict__ zd, int64_t ncols, LenPlan pl, int W, int ld, Mask mask)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R>* bufa = reinterpret_cast<cx<R>*>(smem_raw);
    cx<R>* bufb = bufa + W * ld;
    cx<R>* tws = bufb + W * ld;
    const int Z = pl.L;
    const int64_t c0 = (int64_t)blockIdx.x * W;
    load_twiddles<R>(tws, pl);
    stage_tile<cx<R>>(
        W * Z,
        [&](int idx) {
            const int z = idx / W, w = idx - z * W;
            const int64_t c = c0 + w;
            return c < ncols ? zd[(int64_t)z * ncols + c] : mk<R>(0, 0);
        },
        [&](int idx, cx<R> v) {
            const int z = idx / W, w = idx - z * W;
            bufa[w * ld + z] = v;
        });
    __syncthreads();
    cx<R>* p = smem_fft<-1, R>(bufa, bufb, ld, W, pl, tws);
    cx<R>* q = (p == bufa) ? bufb : bufa;
    for (int idx = threadIdx.x; idx < W * Z; idx += blockDim.x) {
        const int kz = idx / W, w = idx - kz * W;
        const int64_t c = c0 + w;
        if (c < ncols) p[w * ld + kz] = mask(p[w * ld + kz], 0, c, kz);
    }
    __syncthreads();
    cx<R>* r = smem_fft<+1, R>(p, q, ld, W, pl, tws);
    for (int idx = threadIdx.x; idx < W * Z; idx += blockDim.x) {
        const int z = idx / W, w = idx - z * W;
        const int64_t c = c0 + w;
        if (c < ncols) zd[(int64_t)z * ncols + c] = r[w * ld + z];
    }
}

template <typename R, class Mask>
static void launch_zmask(cx<R>* zd, int64_t ncols, const LenPlan& pz, Mask mask, cudaStream_t st)
{
    if constexpr (std::is_same<R, df64>::value) {
        if (!pz.no_reg && line3_length(pz.L)) {
            launch_line3_zmask(zd, ncols, pz, mask, st);
            TTM_LAUNCH_CHECK();
            return;
        }
    }
    const int Z = pz.L;
    const int ld = Z | 1;
    int W = 16;
    while (W > 2 && (2 * (size_t)W * ld + Z) * sizeof(cx<R>) > 110 * 1024) W /= 2;
    const size_t smem = (2 * (size_t)W * ld + Z) * sizeof(cx<R>);
    auto k = k_zmask<R, Mask>;
    set_smem(k, smem);
    k<<<(unsigned)ceil_div(ncols, W), 256, smem, st>>>(zd, ncols, pz, W, ld, mask);
    TTM_LAUNCH_CHECK();
}

__global__ void k_octant_to_df(const double* __restrict__ in, int64_t n, float2* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = in[i];
        const float h = (float)d;
        out[i] = make_float2(h, (float)(d - (double)h));
    }
}

// ---------------------------------------------------------------- host --

void prep_create(ttm_ctx* ctx, Prep& p, int Zt, int Yt, int Xt, int Z, int Y, int X, int tz, int ty, int tx,
                 const ttm_field_params& fp)
{
    TTM_REQUIRE(Zt >= tz && Yt >= ty && Xt >= tx, E_SHAPE, "tomogram smaller than the template");
    TTM_REQUIRE(Zt >= 2 && Yt >= 2 && Xt >= 2, E_SHAPE, "each tomogram axis needs at least 2 voxels");
    TTM_REQUIRE(Z >= Zt && Y >= Yt && X >= Xt, E_SHAPE, "working grid smaller than the tomogram");
    p.Zt = Zt; p.Yt = Yt; p.Xt = Xt;
    p.Z = Z; p.Y = Y; p.X = X; p.Xh = X / 2 + 1;
    p.tz = tz; p.ty = ty; p.tx = tx;
    p.filter_a = fp.filter_a;
    p.px32 = ctx_len_plan(ctx, X, TW_F32);
    p.py32 = ctx_len_plan(ctx, Y, TW_F32);
    p.pz32 = ctx_len_plan(ctx, Z, TW_F32);
    p.px64 = make_len_plan(ctx->twiddles, X, TW_F64);
    p.py64 = make_len_plan(ctx->twiddles, Y, TW_F64);
    p.pz64 = make_len_plan(ctx->twiddles, Z, TW_F64);
    p.pxd = ctx_len_plan(ctx, X, TW_DF64);
    p.pyd = ctx_len_plan(ctx, Y, TW_DF64);
    p.pzd = ctx_len_plan(ctx, Z, TW_DF64);
    const int64_t V = (int64_t)Z * Y * X, Vh = (int64_t)Z * Y * p.Xh;
    p.nblk_pre = prefilter_blocks(Z, Y, X);
    p.g32.alloc(V * sizeof(float));
    p.G.alloc(Vh * sizeof(float2));
    p.zc.alloc(V * sizeof(double2));
    p.w.alloc(V * sizeof(float));
    p.partials.alloc(p.nblk_pre * sizeof(double));
    p.floor.alloc(sizeof(double));
    const int64_t noct = (int64_t)(Z / 2 + 1) * (Y / 2 + 1) * (X / 2 + 1);
    p.mhat.alloc(noct * sizeof(double));

    std::vector<double> m;
    p.M = make_mask(tz, ty, tx, fp.mask_radius, fp.mask_soft_width, m);
    TTM_REQUIRE(p.M > 0, E_INVALID_ARG, "mask is empty");
    p.mask_t.alloc(m.size() * sizeof(double));
    TTM_CUDA_TRY(cudaMemcpy(p.mask_t.p, m.data(), m.size() * sizeof(double), cudaMemcpyHostToDevice));

    // mask spectrum (FP64, once per plan): R2C rows, then y and z passes,
    // using zc as the complex scratch
    cudaStream_t st = 0;
    double2* spec = p.zc.as<double2>();
    SrcWrappedMask src{p.mask_t.as<double>(), Y, X, Z, tz, ty, tx};
    launch_r2c_any<double>(src, (int64_t)Z * Y, spec, p.px64, st);
    launch_strided_any<double, -1>(spec, StridedAxis{p.Xh, Z, (int64_t)Y * p.Xh, p.Xh}, p.py64,
                               ProIdentity<double>(), StoreTo<double>{spec, (int64_t)Y * p.Xh, p.Xh}, st);
    launch_strided_any<double, -1>(spec, StridedAxis{(int64_t)Y * p.Xh, 1, 0, (int64_t)Y * p.Xh}, p.pz64,
                               ProIdentity<double>(), StoreTo<double>{spec, 0, (int64_t)Y * p.Xh}, st);
    k_mhat_octant<<<1024, 256, 0, st>>>(spec, Z, Y, p.Xh, X, 1.0 / (double)V, p.mhat.as<double>());
    TTM_LAUNCH_CHECK();
    p.mhat_df.alloc(noct * sizeof(float2));
    k_octant_to_df<<<1024, 256, 0, st>>>(p.mhat.as<double>(), noct, p.mhat_df.as<float2>());
    TTM_LAUNCH_CHECK();
    TTM_CUDA_TRY(cudaStreamSynchronize(st));
}

void prep_filter(Prep& p, const float* d_tomo, cudaStream_t st)
{
    const int64_t Vt = (int64_t)p.Zt * p.Yt * p.Xt;
    if (p.localsum_mode == 1)
        k_prefilter<true><<<(unsigned)p.nblk_pre, kPreThreads, 0, st>>>(
            d_tomo, p.Zt, p.Yt, p.Xt, p.Z, p.Y, p.X, (float)p.filter_a, p.g32.as<float>(),
            localsum_reads_g(p) ? nullptr : p.zc.as<double2>(), p.partials.as<double>());
    else
        k_prefilter<false><<<(unsigned)p.nblk_pre, kPreThreads, 0, st>>>(d_tomo, p.Zt, p.Yt, p.Xt, p.Z, p.Y, p.X,
                                                                      (float)p.filter_a, p.g32.as<float>(),
                                                                      p.zc.as<double2>(), p.partials.as<double>());
    TTM_LAUNCH_CHECK();
    k_var_floor<<<1, 1024, 0, st>>>(p.partials.as<double>(), p.nblk_pre, Vt, p.M, p.floor.as<double>());
    TTM_LAUNCH_CHECK();
}

// G = FFT(g): x (real-to-complex), y, z
void prep_spectrum(Prep& p, cudaStream_t st)
{
    const int Z = p.Z, Y = p.Y, X = p.X, Xh = p.Xh;
    float2* G = p.G.as<float2>();
    launch_r2c_any<float>(SrcFloat{p.g32.as<float>(), X}, (int64_t)Z * Y, G, p.px32, st);
    launch_strided_any<float, -1>(G, StridedAxis{Xh, Z, (int64_t)Y * Xh, Xh}, p.py32, ProIdentity<float>(),
                              StoreTo<float>{G, (int64_t)Y * Xh, Xh}, st);
    launch_strided_any<float, -1>(G, StridedAxis{(int64_t)Y * Xh, 1, 0, (int64_t)Y * Xh}, p.pz32,
                              ProIdentity<float>(), StoreTo<float>{G, 0, (int64_t)Y * Xh}, st);
}

// local sums: forward x, y of (g + i g^2), the fused z pass (forward,
// times the mask spectrum, inverse), inverse y, x with the w epilogue; in
// FP64 or in double-float
void prep_localsums(Prep& p, cudaStream_t st)
{
    const int Z = p.Z, Y = p.Y, X = p.X;
    const int64_t YX = (int64_t)Y * X;
    if (p.localsum_mode == 1) {
        dcx* zd = p.zc.as<dcx>();
        if (localsum_reads_g(p))
            launch_line3_contig_src<-1>((int64_t)Z * Y, p.pxd, SrcGSquared{p.g32.as<float>(), X},
                                        StoreTo<df64>{zd, X, 1}, st);
        else
            launch_contig_any<df64, -1>(zd, (int64_t)Z * Y, p.pxd, ProIdentity<df64>(), StoreTo<df64>{zd, X, 1},
                                        st);
        TTM_LAUNCH_CHECK();
        launch_strided_any<df64, -1>(zd, StridedAxis{X, Z, YX, X}, p.pyd, ProIdentity<df64>(),
                                     StoreTo<df64>{zd, YX, X}, st);
        launch_zmask<df64>(zd, YX, p.pzd, ProMaskSpectrumDF{p.mhat_df.as<float2>(), Z, Y, X}, st);
        launch_strided_any<df64, +1>(zd, StridedAxis{X, Z, YX, X}, p.pyd, ProIdentity<df64>(),
                                     StoreTo<df64>{zd, YX, X}, st);
        launch_contig_any<df64, +1>(zd, (int64_t)Z * Y, p.pxd, ProIdentity<df64>(),
                                    StoreWDF{p.w.as<float>(), p.floor.as<double>(), df64(1.0 / p.M), X}, st);
        return;
    }
    double2* zc = p.zc.as<double2>();
    launch_contig_any<double, -1>(zc, (int64_t)Z * Y, p.px64, ProIdentity<double>(), StoreTo<double>{zc, X, 1}, st);
    launch_strided_any<double, -1>(zc, StridedAxis{X, Z, YX, X}, p.py64, ProIdentity<double>(),
                                   StoreTo<double>{zc, YX, X}, st);
    launch_zmask<double>(zc, YX, p.pz64, ProMaskSpectrum{p.mhat.as<double>(), Z, Y, X}, st);
    launch_strided_any<double, +1>(zc, StridedAxis{X, Z, YX, X}, p.py64, ProIdentity<double>(),
                                   StoreTo<double>{zc, YX, X}, st);
    launch_contig_any<double, +1>(zc, (int64_t)Z * Y, p.px64, ProIdentity<double>(),
                                  StoreW{p.w.as<float>(), p.floor.as<double>(), p.M, X}, st);
}

}  // namespace ttm
