// fft.cuh -- batched 1-D FFT passes over one axis of a 3-D array.
//
// Each CTA stages a tile of W lines of length L in shared memory, runs a
// mixed-radix Stockham FFT (radices 2, 3, 4, 5, 7, 8; the autosort variant
// so no bit reversal is needed) through two ping-pong buffers, and writes
// the tile back. Tiles of a strided axis are W lines that are adjacent in
// memory, so every one of the L rows of the tile is a contiguous run of W
// complex elements (coalesced); tiles of the contiguous axis are W whole
// lines. Loads go through a "prologue" functor and stores through a "store"
// functor, which is how the pointwise spectrum products, the real<->complex
// packing and the normalisation epilogues are fused into the passes.
//
// Direction DIR = -1 computes sum_j x_j exp(-2 pi i jk/L) (forward),
// DIR = +1 the unnormalised inverse.
#pragma once

#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ttm_common.cuh"
#include "df64.cuh"

namespace ttm {

// Complex values as stored in HBM: the pass precision itself, or FP16 /
// BF16 pairs that are widened to FP32 on load (the arithmetic stays FP32).
__device__ __forceinline__ float2 load_cx(const float2& v) { return v; }
__device__ __forceinline__ double2 load_cx(const double2& v) { return v; }
__device__ __forceinline__ dcx load_cx(const dcx& v) { return v; }
__device__ __forceinline__ float2 load_cx(const __half2& v) { return __half22float2(v); }
__device__ __forceinline__ float2 load_cx(const __nv_bfloat162& v) { return __bfloat1622float2(v); }
__device__ __forceinline__ void store_cx(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void store_cx(__half2* p, float2 v) { *p = __float22half2_rn(v); }
__device__ __forceinline__ void store_cx(__nv_bfloat162* p, float2 v) { *p = __float22bfloat162_rn(v); }

constexpr int kMaxStages = 24;

// A transform length with its radix schedule and its twiddle table
// tw[m] = exp(-2 pi i m / L), m in [0, L), in the pass precision.
struct LenPlan {
    int L;
    int nst;
    int rad[kMaxStages];
    const void* tw;
    int tile_w = 0;   // lines per CTA of the shared-memory passes (0: default)
    int no_reg = 0;   // 1: use the shared-memory passes even where register kernels exist
};

// sin/cos of 2 pi m / R for the odd radices (mathematical constants)
struct OddRadixConst {
    static constexpr double c3 = -0.5;
    static constexpr double s3 = 0.86602540378443864676372317075294;
    static constexpr double c5_1 = 0.30901699437494742410229341718282;
    static constexpr double s5_1 = 0.95105651629515357211643933337938;
    static constexpr double c5_2 = -0.80901699437494742410229341718282;
    static constexpr double s5_2 = 0.58778525229247312916870595463907;
    static constexpr double c7_1 = 0.62348980185873353052500488400424;
    static constexpr double s7_1 = 0.78183148246802980870844452667406;
    static constexpr double c7_2 = -0.22252093395631440428890256449679;
    static constexpr double s7_2 = 0.97492791218182360701813168299393;
    static constexpr double c7_3 = -0.90096886790241912623610231950745;
    static constexpr double s7_3 = 0.43388373911755812047576833284836;
    static constexpr double sqrt_half = 0.70710678118654752440084436210485;
};

// ---------------------------------------------------------- butterflies --

template <int DIR, typename C> __device__ __forceinline__ void dft2(C* v)
{
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <int DIR, typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3)
{
    C t0 = cadd(a0, a2), t1 = csub(a0, a2);
    C t2 = cadd(a1, a3), t3 = cmul_diri<DIR>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

// x * (h + DIR h i) = h (x.x - DIR x.y) + i h (x.y + DIR x.x): two adds and
// two products instead of a full complex product
template <int DIR, typename R> __device__ __forceinline__ cx<R> mul_w8_1(cx<R> x, R h)
{
    return DIR < 0 ? mk<R>((x.x + x.y) * h, (x.y - x.x) * h) : mk<R>((x.x - x.y) * h, (x.y + x.x) * h);
}
// x * (-h + DIR h i) = h (-x.x - DIR x.y) + i h (DIR x.x - x.y)
template <int DIR, typename R> __device__ __forceinline__ cx<R> mul_w8_3(cx<R> x, R h)
{
    return DIR < 0 ? mk<R>((x.y - x.x) * h, (-x.x - x.y) * h) : mk<R>((-x.x - x.y) * h, (x.x - x.y) * h);
}

template <int DIR, typename R> __device__ __forceinline__ void dft8(cx<R>* v)
{
    cx<R> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    cx<R> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<DIR>(e0, e1, e2, e3);
    dft4<DIR>(o0, o1, o2, o3);
    const R h = (R)OddRadixConst::sqrt_half;
    // w8^1 = h(1 + DIR i), w8^2 = DIR i, w8^3 = h(-1 + DIR i)
    cx<R> t1 = mul_w8_1<DIR, R>(o1, h);
    cx<R> t2 = cmul_diri<DIR>(o2);
    cx<R> t3 = mul_w8_3<DIR, R>(o3, h);
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, t1); v[5] = csub(e1, t1);
    v[2] = cadd(e2, t2); v[6] = csub(e2, t2);
    v[3] = cadd(e3, t3); v[7] = csub(e3, t3);
}

// Odd radices in their symmetric form: with t_r = x_r + x_{R-r} and
// d_r = x_r - x_{R-r} (r = 1..(R-1)/2),
//   X_0 = x_0 + sum_r t_r,
//   X_k, X_{R-k} = A_k +- DIR i B_k,  A_k = x_0 + sum_r t_r cos(2 pi rk/R),
//                                      B_k = sum_r d_r sin(2 pi rk/R),
// so every product is a real constant times a complex value and each
// cosine / sine term is shared by the output pair (k, R - k).
template <int DIR, typename R> __device__ __forceinline__ cx<R> pm_diri(cx<R> a, cx<R> b, bool plus)
{
    // a + DIR i b (plus) or a - DIR i b
    const cx<R> ib = cmul_diri<DIR>(b);
    return plus ? cadd(a, ib) : csub(a, ib);
}

template <int DIR, typename R> __device__ __forceinline__ void dft3(cx<R>* v)
{
    const cx<R> t = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    const cx<R> x0 = v[0];
    v[0] = cadd(x0, t);
    const cx<R> A = csub(x0, cscale(t, (R)0.5));
    const cx<R> B = cscale(d, (R)OddRadixConst::s3);
    v[1] = pm_diri<DIR, R>(A, B, true);
    v[2] = pm_diri<DIR, R>(A, B, false);
}

template <int DIR, typename R> __device__ __forceinline__ void dft5(cx<R>* v)
{
    const R c1 = (R)OddRadixConst::c5_1, c2 = (R)OddRadixConst::c5_2;
    const R s1 = (R)OddRadixConst::s5_1, s2 = (R)OddRadixConst::s5_2;
    const cx<R> x0 = v[0];
    const cx<R> t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    const cx<R> d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
    v[0] = cadd(x0, cadd(t1, t2));
    // cos 4 pi/5 = c2, cos 8 pi/5 = c1; sin 8 pi/5 = -s1
    const cx<R> A1 = cadd(x0, cadd(cscale(t1, c1), cscale(t2, c2)));
    const cx<R> A2 = cadd(x0, cadd(cscale(t1, c2), cscale(t2, c1)));
    const cx<R> B1 = cadd(cscale(d1, s1), cscale(d2, s2));
    const cx<R> B2 = csub(cscale(d1, s2), cscale(d2, s1));
    v[1] = pm_diri<DIR, R>(A1, B1, true);
    v[4] = pm_diri<DIR, R>(A1, B1, false);
    v[2] = pm_diri<DIR, R>(A2, B2, true);
    v[3] = pm_diri<DIR, R>(A2, B2, false);
}

template <int DIR, typename R> __device__ __forceinline__ void dft7(cx<R>* v)
{
    const R c1 = (R)OddRadixConst::c7_1, c2 = (R)OddRadixConst::c7_2, c3 = (R)OddRadixConst::c7_3;
    const R s1 = (R)OddRadixConst::s7_1, s2 = (R)OddRadixConst::s7_2, s3 = (R)OddRadixConst::s7_3;
    const cx<R> x0 = v[0];
    const cx<R> t1 = cadd(v[1], v[6]), t2 = cadd(v[2], v[5]), t3 = cadd(v[3], v[4]);
    const cx<R> d1 = csub(v[1], v[6]), d2 = csub(v[2], v[5]), d3 = csub(v[3], v[4]);
    v[0] = cadd(x0, cadd(t1, cadd(t2, t3)));
    // angles 2 pi rk / 7 reduced: (r k mod 7) in {1,2,3} keeps its sine, in
    // {4,5,6} takes minus the sine of 7 - (r k mod 7)
    const cx<R> A1 = cadd(x0, cadd(cscale(t1, c1), cadd(cscale(t2, c2), cscale(t3, c3))));
    const cx<R> A2 = cadd(x0, cadd(cscale(t1, c2), cadd(cscale(t2, c3), cscale(t3, c1))));
    const cx<R> A3 = cadd(x0, cadd(cscale(t1, c3), cadd(cscale(t2, c1), cscale(t3, c2))));
    const cx<R> B1 = cadd(cscale(d1, s1), cadd(cscale(d2, s2), cscale(d3, s3)));
    const cx<R> B2 = csub(cscale(d1, s2), cadd(cscale(d2, s3), cscale(d3, s1)));
    const cx<R> B3 = cadd(csub(cscale(d1, s3), cscale(d2, s1)), cscale(d3, s2));
    v[1] = pm_diri<DIR, R>(A1, B1, true);
    v[6] = pm_diri<DIR, R>(A1, B1, false);
    v[2] = pm_diri<DIR, R>(A2, B2, true);
    v[5] = pm_diri<DIR, R>(A2, B2, false);
    v[3] = pm_diri<DIR, R>(A3, B3, true);
    v[4] = pm_diri<DIR, R>(A3, B3, false);
}

template <int RAD, int DIR, typename R> __device__ __forceinline__ void dft(cx<R>* v)
{
    if constexpr (RAD == 2) dft2<DIR>(v);
    else if constexpr (RAD == 3) dft3<DIR, R>(v);
    else if constexpr (RAD == 4) dft4<DIR>(v[0], v[1], v[2], v[3]);
    else if constexpr (RAD == 5) dft5<DIR, R>(v);
    else if constexpr (RAD == 7) dft7<DIR, R>(v);
    else dft8<DIR, R>(v);
    // double-float butterflies add without renormalising (df64.cuh): once
    // per output here
    if constexpr (std::is_same<R, df64>::value) {
#pragma unroll
        for (int r = 0; r < RAD; r++) v[r] = renormalise(v[r]);
    }
}

// ----------------------------------------------------------- stages --

// One Stockham stage of radix RAD on W lines (line stride ld) from `in` to
// `out`. Ns = product of the radices of the earlier stages.
template <int RAD, int DIR, typename R>
__device__ __forceinline__ void stockham_stage(const cx<R>* __restrict__ in, cx<R>* __restrict__ out,
                                               int L, int ld, int W, int Ns,
                                               const cx<R>* __restrict__ tw)
{
    const int nb = L / RAD;
    const int total = nb * W;
    const int step = L / (Ns * RAD);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        int w = t / nb;
        int j = t - w * nb;
        int k = j % Ns;
        const cx<R>* src = in + w * ld;
        cx<R> v[RAD];
#pragma unroll
        for (int r = 0; r < RAD; r++) v[r] = src[j + r * nb];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < RAD; r++) {
                cx<R> t_ = tw[r * k * step];
                if (DIR > 0) t_.y = -t_.y;
                v[r] = cmul(v[r], t_);
            }
        }
        dft<RAD, DIR, R>(v);
        cx<R>* dst = out + w * ld;
        int base = (j / Ns) * Ns * RAD + k;
#pragma unroll
        for (int r = 0; r < RAD; r++) dst[base + r * Ns] = v[r];
    }
}

// Full transform of the W lines in a (scratch b); returns the buffer that
// holds the result. Ends with __syncthreads().
template <int DIR, typename R>
__device__ cx<R>* smem_fft(cx<R>* a, cx<R>* b, int ld, int W, const LenPlan& pl, const cx<R>* tw)
{
    int Ns = 1;
    const int L = pl.L;
    for (int s = 0; s < pl.nst; s++) {
        switch (pl.rad[s]) {
            case 2: stockham_stage<2, DIR, R>(a, b, L, ld, W, Ns, tw); break;
            case 3: stockham_stage<3, DIR, R>(a, b, L, ld, W, Ns, tw); break;
            case 4: stockham_stage<4, DIR, R>(a, b, L, ld, W, Ns, tw); break;
            case 5: stockham_stage<5, DIR, R>(a, b, L, ld, W, Ns, tw); break;
            case 7: stockham_stage<7, DIR, R>(a, b, L, ld, W, Ns, tw); break;
            default: stockham_stage<8, DIR, R>(a, b, L, ld, W, Ns, tw); break;
        }
        Ns *= pl.rad[s];
        __syncthreads();
        cx<R>* t = a; a = b; b = t;
    }
    return a;
}

template <typename R>
__device__ __forceinline__ void load_twiddles(cx<R>* tws, const LenPlan& pl)
{
    const cx<R>* g = reinterpret_cast<const cx<R>*>(pl.tw);
    for (int i = threadIdx.x; i < pl.L; i += blockDim.x) tws[i] = g[i];
}

// Stages n tile elements into shared memory with kLoadBatch global loads
// per thread issued before any of their shared-memory stores, so that a
// thread has that many loads in flight instead of waiting on each in turn:
// get(idx) loads element idx, put(idx, v) stores it into the tile.
constexpr int kLoadBatch = 8;
template <typename T, class Get, class Put>
__device__ __forceinline__ void stage_tile(int n, Get get, Put put)
{
    for (int base = threadIdx.x; base < n; base += kLoadBatch * blockDim.x) {
        T v[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; u++) {
            const int idx = base + u * (int)blockDim.x;
            if (idx < n) v[u] = get(idx);
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; u++) {
            const int idx = base + u * (int)blockDim.x;
            if (idx < n) put(idx, v[u]);
        }
    }
}

// ------------------------------------------------------------ functors --

template <typename R> struct ProIdentity {
    __device__ __forceinline__ cx<R> operator()(cx<R> v, int64_t, int64_t, int) const { return v; }
};

template <typename R> struct StoreTo {
    cx<R>* out;
    int64_t os, s;  // outer stride, element stride (inner stride is 1)
    __device__ __forceinline__ void operator()(cx<R> v, int64_t o, int64_t i, int j) const
    {
        out[o * os + i + (int64_t)j * s] = v;
    }
};

// Geometry of a strided axis: line (o, i) has elements o*os + i + j*s,
// j < L; i < inner are adjacent lines, o < outer.
struct StridedAxis {
    int64_t inner, outer, os, s;
};

// ------------------------------------------------------------ kernels --

// Shared memory: 2 * W * ld + L complex elements.
template <typename R, int DIR, class Pro, class Store, typename In = cx<R>>
__global__ void __launch_bounds__(256) k_fft_strided(const In* __restrict__ in, StridedAxis ax, LenPlan pl,
                                                     int W, int ld, Pro pro, Store store)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R>* bufa = reinterpret_cast<cx<R>*>(smem_raw);
    cx<R>* bufb = bufa + W * ld;
    cx<R>* tws = bufb + W * ld;
    const int64_t tiles_per_outer = (ax.inner + W - 1) / W;
    const int64_t o = blockIdx.x / tiles_per_outer;
    const int64_t i0 = (blockIdx.x - o * tiles_per_outer) * W;
    const int L = pl.L;
    load_twiddles<R>(tws, pl);
    stage_tile<cx<R>>(
        W * L,
        [&](int idx) {
            const int j = idx / W, w = idx - j * W;
            const int64_t i = i0 + w;
            return i < ax.inner ? pro(load_cx(in[o * ax.os + i + (int64_t)j * ax.s]), o, i, j) : mk<R>(0, 0);
        },
        [&](int idx, cx<R> v) {
            const int j = idx / W, w = idx - j * W;
            bufa[w * ld + j] = v;
        });
    __syncthreads();
    cx<R>* res = smem_fft<DIR, R>(bufa, bufb, ld, W, pl, tws);
    for (int idx = threadIdx.x; idx < W * L; idx += blockDim.x) {
        int j = idx / W, w = idx - j * W;
        int64_t i = i0 + w;
        if (i < ax.inner) store(res[w * ld + j], o, i, j);
    }
}

// Contiguous lines: line l has elements l*L + j (l < nlines). The functors
// get (o = l, i = 0, j).
template <typename R, int DIR, class Pro, class Store>
__global__ void __launch_bounds__(256) k_fft_contig(const cx<R>* __restrict__ in, int64_t nlines, LenPlan pl,
                                                    int W, int ld, Pro pro, Store store)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R>* bufa = reinterpret_cast<cx<R>*>(smem_raw);
    cx<R>* bufb = bufa + W * ld;
    cx<R>* tws = bufb + W * ld;
    const int64_t l0 = (int64_t)blockIdx.x * W;
    const int L = pl.L;
    load_twiddles<R>(tws, pl);
    stage_tile<cx<R>>(
        W * L,
        [&](int idx) {
            const int w = idx / L, j = idx - w * L;
            const int64_t l = l0 + w;
            return l < nlines ? pro(in[l * L + j], l, 0, j) : mk<R>(0, 0);
        },
        [&](int idx, cx<R> v) {
            const int w = idx / L, j = idx - w * L;
            bufa[w * ld + j] = v;
        });
    __syncthreads();
    cx<R>* res = smem_fft<DIR, R>(bufa, bufb, ld, W, pl, tws);
    for (int idx = threadIdx.x; idx < W * L; idx += blockDim.x) {
        int w = idx / L, j = idx - w * L;
        int64_t l = l0 + w;
        if (l < nlines) store(res[w * ld + j], l, 0, j);
    }
}

// Forward real-to-complex along the contiguous axis, two real rows per
// complex line: z = a + i b, Z = FFT(z), A(k) = (Z(k) + conj Z(-k)) / 2,
// B(k) = (Z(k) - conj Z(-k)) / (2i), k in [0, X/2]. `src(row, x)` yields the
// real input (so padding / wrapping / type conversion fuse into the load).
template <typename R, class Src>
__global__ void __launch_bounds__(256) k_r2c_rows(Src src, int64_t nrows, cx<R>* __restrict__ out, LenPlan pl,
                                                  int W, int ld)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R>* bufa = reinterpret_cast<cx<R>*>(smem_raw);
    cx<R>* bufb = bufa + W * ld;
    cx<R>* tws = bufb + W * ld;
    const int X = pl.L, Xh = X / 2 + 1;
    const int64_t r0 = (int64_t)blockIdx.x * 2 * W;
    load_twiddles<R>(tws, pl);
    for (int idx = threadIdx.x; idx < W * X; idx += blockDim.x) {
        int w = idx / X, x = idx - w * X;
        int64_t ra = r0 + 2 * w, rb = ra + 1;
        R a = ra < nrows ? src(ra, x) : (R)0;
        R b = rb < nrows ? src(rb, x) : (R)0;
        bufa[w * ld + x] = mk<R>(a, b);
    }
    __syncthreads();
    cx<R>* res = smem_fft<-1, R>(bufa, bufb, ld, W, pl, tws);
    for (int idx = threadIdx.x; idx < W * Xh; idx += blockDim.x) {
        int w = idx / Xh, k = idx - w * Xh;
        int64_t ra = r0 + 2 * w, rb = ra + 1;
        cx<R> zk = res[w * ld + k];
        cx<R> zn = res[w * ld + (k == 0 ? 0 : X - k)];
        // A = (zk + conj zn)/2 ; B = (zk - conj zn)/(2i)
        cx<R> A = mk<R>((zk.x + zn.x) * (R)0.5, (zk.y - zn.y) * (R)0.5);
        cx<R> d = mk<R>(zk.x - zn.x, zk.y + zn.y);
        cx<R> B = mk<R>(d.y * (R)0.5, -d.x * (R)0.5);
        if (ra < nrows) out[ra * Xh + k] = A;
        if (rb < nrows) out[rb * Xh + k] = B;
    }
}

// Inverse complex-to-real along the contiguous axis, two half-spectrum rows
// per complex line: Z(k) = A(k) + i B(k) for k <= X/2 and
// Z(k) = conj A(X-k) + i conj B(X-k) above, with the imaginary parts of the
// k = 0 (and k = X/2 for even X) bins dropped as a C2R transform does;
// IFFT(Z) = a + i b. `sink(row, x, value)` consumes the real outputs
// (normalisation / max epilogues). `in` may be offset per blockIdx.y by
// in_batch_stride for batched use; the sink gets blockIdx.y via `batch`.
template <typename R, class Sink, typename In = cx<R>>
__global__ void __launch_bounds__(256) k_c2r_rows(const In* __restrict__ in, int64_t nrows, Sink sink,
                                                  LenPlan pl, int W, int ld, int nbatch)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R>* bufa = reinterpret_cast<cx<R>*>(smem_raw);
    cx<R>* bufb = bufa + W * ld;
    cx<R>* tws = bufb + W * ld;
    const int X = pl.L, Xh = X / 2 + 1;
    // batch index fastest so that the CTAs sharing rows (and the rows of any
    // per-voxel factor the sink reads) run together
    const int batch = blockIdx.x % nbatch;
    const int64_t tile = blockIdx.x / nbatch;
    const int64_t r0 = tile * 2 * W;
    const In* src = in + (int64_t)batch * nrows * Xh;
    load_twiddles<R>(tws, pl);
    for (int idx = threadIdx.x; idx < W * Xh; idx += blockDim.x) {
        int w = idx / Xh, k = idx - w * Xh;
        int64_t ra = r0 + 2 * w, rb = ra + 1;
        cx<R> A = ra < nrows ? load_cx(src[ra * Xh + k]) : mk<R>(0, 0);
        cx<R> B = rb < nrows ? load_cx(src[rb * Xh + k]) : mk<R>(0, 0);
        if (k == 0 || (2 * k == X)) { A.y = 0; B.y = 0; }
        // Z(k) = A + iB
        bufa[w * ld + k] = mk<R>(A.x - B.y, A.y + B.x);
        // Z(X-k) = conj A + i conj B, for the bins not covered above
        int kk = X - k;
        if (k >= 1 && kk >= Xh) bufa[w * ld + kk] = mk<R>(A.x + B.y, -A.y + B.x);
    }
    __syncthreads();
    cx<R>* res = smem_fft<+1, R>(bufa, bufb, ld, W, pl, tws);
    for (int idx = threadIdx.x; idx < W * X; idx += blockDim.x) {
        int w = idx / X, x = idx - w * X;
        int64_t ra = r0 + 2 * w, rb = ra + 1;
        cx<R> v = res[w * ld + x];
        if (ra < nrows) sink(batch, ra, x, v.x);
        if (rb < nrows) sink(batch, rb, x, v.y);
    }
}

// ------------------------------------------------------------ host side --

// Radix schedule for L (7-smooth); returns false otherwise.
bool factor_length(int L, LenPlan& pl);

// Tile width (lines per CTA) and padded line stride for a pass of length L
// in precision R, and its dynamic shared memory in bytes.
struct TileShape {
    int W, ld;
    size_t smem;
};
TileShape choose_tile(int L, size_t elem_bytes, int min_w, int max_w);
// the plan's tuned tile width if it has one (within the shared-memory
// budget), else choose_tile
TileShape plan_tile(const LenPlan& pl, size_t elem_bytes, int min_w, int max_w);

}  // namespace ttm

namespace ttm {

// Device twiddle tables, one per (length, precision), owned by a context.
// twiddle precision: FP32, FP64, or double-float pairs
enum TwKind { TW_F32 = 0, TW_F64 = 1, TW_DF64 = 2 };

class TwiddleCache {
  public:
    ~TwiddleCache();
    const void* get(int L, int kind);

  private:
    struct Entry { int L; int kind; void* ptr; };
    Entry* entries_ = nullptr;
    int n_ = 0, cap_ = 0;
};

// LenPlan for L with the twiddles of the given precision (TwKind).
LenPlan make_len_plan(TwiddleCache& tc, int L, int kind);

template <typename K>
inline void set_smem(K kernel, size_t bytes)
{
    if (bytes > 48 * 1024)
        TTM_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

// strided-axis pass (lines adjacent along the inner index)
template <typename R, int DIR, class Pro, class Store, typename In = cx<R>>
inline void launch_strided(const In* in, StridedAxis ax, const LenPlan& pl, Pro pro, Store store,
                           cudaStream_t st)
{
    TileShape ts = plan_tile(pl, sizeof(cx<R>), 4, 16);
    auto k = k_fft_strided<R, DIR, Pro, Store, In>;
    set_smem(k, ts.smem);
    int64_t grid = ax.outer * ceil_div(ax.inner, ts.W);
    TTM_REQUIRE(grid < (1ll << 31), E_SHAPE, "strided pass grid too large");
    k<<<(unsigned)grid, 256, ts.smem, st>>>(in, ax, pl, ts.W, ts.ld, pro, store);
    TTM_LAUNCH_CHECK();
}

template <typename R, int DIR, class Pro, class Store>
inline void launch_contig(const cx<R>* in, int64_t nlines, const LenPlan& pl, Pro pro, Store store,
                          cudaStream_t st)
{
    TileShape ts = plan_tile(pl, sizeof(cx<R>), 1, 8);
    auto k = k_fft_contig<R, DIR, Pro, Store>;
    set_smem(k, ts.smem);
    int64_t grid = ceil_div(nlines, ts.W);
    k<<<(unsigned)grid, 256, ts.smem, st>>>(in, nlines, pl, ts.W, ts.ld, pro, store);
    TTM_LAUNCH_CHECK();
}

template <typename R, class Src>
inline void launch_r2c_rows(Src src, int64_t nrows, cx<R>* out, const LenPlan& pl, cudaStream_t st)
{
    TileShape ts = choose_tile(pl.L, sizeof(cx<R>), 1, 8);
    auto k = k_r2c_rows<R, Src>;
    set_smem(k, ts.smem);
    int64_t grid = ceil_div(nrows, 2 * ts.W);
    k<<<(unsigned)grid, 256, ts.smem, st>>>(src, nrows, out, pl, ts.W, ts.ld);
    TTM_LAUNCH_CHECK();
}

template <typename R, class Sink, typename In = cx<R>>
inline void launch_c2r_rows(const In* in, int64_t nrows, Sink sink, const LenPlan& pl, int nbatch,
                            cudaStream_t st)
{
    TileShape ts = plan_tile(pl, sizeof(cx<R>), 1, 8);
    auto k = k_c2r_rows<R, Sink, In>;
    set_smem(k, ts.smem);
    int64_t grid = ceil_div(nrows, 2 * ts.W) * nbatch;
    TTM_REQUIRE(grid < (1ll << 31), E_SHAPE, "c2r pass grid too large");
    k<<<(unsigned)grid, 256, ts.smem, st>>>(in, nrows, sink, pl, ts.W, ts.ld, nbatch);
    TTM_LAUNCH_CHECK();
}

}  // namespace ttm
