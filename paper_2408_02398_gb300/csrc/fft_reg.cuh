// fft_reg.cuh -- register-resident FFT passes for the lengths the hot path
// uses most (L = E * P with P | E, E <= 32).
//
// Four-step decomposition of one line, L = E * P, input index j = p + P m,
// output index k = k1 + E k2:
//   X[k1 + E k2] = sum_p w_P^{p k2} [ w_L^{p k1} sum_m x[p + P m] w_E^{m k1} ]
// Thread p of a line holds its E inputs in registers, does the E-point DFT
// and the twiddles in registers, one shared-memory transpose hands each
// thread the P values of E/P columns k1, and the P-point DFTs finish in
// registers. Running the same steps backwards with conjugated twiddles gives
// the inverse transform from the (k1 + E k2) layout straight back to the
// natural layout, which the fused z pass uses to multiply spectra without a
// second transpose. Small DFTs are themselves split recursively into the
// radices 2, 3, 4, 5, 7, 8 with compile-time twiddle indices into the
// length-L table exp(-2 pi i t / L) held in shared memory.
#pragma once

#include <type_traits>

#include "fft.cuh"
#include "fft_line3.cuh"

namespace ttm {

__host__ __device__ constexpr bool is_base_radix(int S) { return S == 2 || S == 3 || S == 4 || S == 5 || S == 7 || S == 8; }
__host__ __device__ constexpr int pick_radix(int S)
{
    return (S % 8 == 0 && S / 8 >= 2) ? 8 : (S % 4 == 0 && S / 4 >= 2) ? 4 : (S % 2 == 0 && S / 2 >= 2) ? 2
         : (S % 5 == 0 && S / 5 >= 2) ? 5 : (S % 3 == 0 && S / 3 >= 2) ? 3 : 7;
}

template <int DIR, typename R>
__device__ __forceinline__ cx<R> twid(const cx<R>* __restrict__ tw, int t)
{
    cx<R> w = tw[t];
    if (DIR > 0) w.y = -w.y;
    return w;
}

// in-place S-point DFT of v (natural order in and out); tw = exp(-2 pi i t / TWL)
template <int S, int DIR, int TWL, typename R>
__device__ __forceinline__ void dft_reg(cx<R>* v, const cx<R>* __restrict__ tw)
{
    if constexpr (S == 1) {
        return;
    } else if constexpr (is_base_radix(S)) {
        dft<S, DIR, R>(v);
    } else {
        constexpr int S1 = pick_radix(S);
        constexpr int S2 = S / S1;
        static_assert(TWL % S == 0, "twiddle table length must be a multiple of S");
        cx<R> T[S1][S2];
#pragma unroll
        for (int p1 = 0; p1 < S1; p1++) {
            cx<R> t[S2];
#pragma unroll
            for (int m = 0; m < S2; m++) t[m] = v[p1 + S1 * m];
            dft_reg<S2, DIR, TWL, R>(t, tw);
#pragma unroll
            for (int k1 = 0; k1 < S2; k1++) {
                if (p1 * k1 != 0) t[k1] = cmul(t[k1], twid<DIR, R>(tw, p1 * k1 * (TWL / S)));
                T[p1][k1] = t[k1];
            }
        }
#pragma unroll
        for (int k1 = 0; k1 < S2; k1++) {
            cx<R> u[S1];
#pragma unroll
            for (int p1 = 0; p1 < S1; p1++) u[p1] = T[p1][k1];
            dft<S1, DIR, R>(u);
#pragma unroll
            for (int k2 = 0; k2 < S1; k2++) v[k1 + S2 * k2] = u[k2];
        }
    }
}

// thread counts and shared-memory layout of a four-step tile of W lines
template <typename R> struct FsThreads { static constexpr int value = 256; };
template <> struct FsThreads<double> { static constexpr int value = 128; };
template <> struct FsThreads<df64> { static constexpr int value = 128; };

template <typename R, int E, int P> struct FsShape {
    static constexpr int L = E * P;
    static constexpr int W = FsThreads<R>::value / P;    // lines per CTA
    static constexpr int KS = P + 1;                     // padded stride of k1 in the transpose
    static constexpr int LD = (E * KS) | 1;              // odd line stride
    static constexpr int THREADS = W * P;
    // twiddles + one transpose buffer
    static constexpr size_t SMEM = ((size_t)L + (size_t)W * LD) * sizeof(cx<R>);
};

template <typename R>
__device__ __forceinline__ void fs_load_tw(cx<R>* tw, const void* g, int L)
{
    const cx<R>* src = reinterpret_cast<const cx<R>*>(g);
    for (int k = threadIdx.x; k < L; k += blockDim.x) tw[k] = src[k];
}

// phase 1 of the forward four-step: E-point DFT + twiddles, then the
// transposed write xch[k1 * KS + p] (xch = this line's buffer)
template <typename R, int E, int P, int DIR>
__device__ __forceinline__ void fs_phase1(cx<R>* x, int p, cx<R>* xch, const cx<R>* tw)
{
    using S = FsShape<R, E, P>;
    dft_reg<E, DIR, S::L, R>(x, tw);
#pragma unroll
    for (int k1 = 1; k1 < E; k1++) x[k1] = cmul(x[k1], twid<DIR, R>(tw, p * k1));
#pragma unroll
    for (int k1 = 0; k1 < E; k1++) xch[k1 * S::KS + p] = x[k1];
}

// --------------------------------------------------------------- passes --

// strided axis: lines (o, i), i adjacent (w fastest in the CTA), elements
// at o*os + i + j*s. Natural order in and out.
template <typename R, int E, int P, int DIR, class Pro, class Store, typename In = cx<R>>
__global__ void __launch_bounds__(FsThreads<R>::value)
k_fs_strided(const In* __restrict__ in, StridedAxis ax, const void* twg, Pro pro, Store store)
{
    using S = FsShape<R, E, P>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R>* tw = reinterpret_cast<cx<R>*>(smem_raw);
    cx<R>* xa = tw + S::L;
    const int t = threadIdx.x;
    const int w = t % S::W, p = t / S::W;
    const int64_t tiles = (ax.inner + S::W - 1) / S::W;
    const int64_t o = blockIdx.x / tiles;
    const int64_t i = (blockIdx.x - o * tiles) * S::W + w;
    const bool act = i < ax.inner;
    fs_load_tw<R>(tw, twg, S::L);
    cx<R> x[E];
    const In* src = in + o * ax.os + i;
#pragma unroll
    for (int m = 0; m < E; m++) {
        const int j = p + P * m;
        x[m] = act ? pro(load_cx(src[(int64_t)j * ax.s]), o, i, j) : mk<R>(0, 0);
    }
    __syncthreads();
    fs_phase1<R, E, P, DIR>(x, p, xa + w * S::LD, tw);
    __syncthreads();
    auto column = [&](int ii) {
        const int k1 = p + P * ii;
        cx<R> u[P];
#pragma unroll
        for (int q = 0; q < P; q++) u[q] = xa[w * S::LD + k1 * S::KS + q];
        dft_reg<P, DIR, S::L, R>(u, tw);
        if (act) {
#pragma unroll
            for (int k2 = 0; k2 < P; k2++) store(u[k2], o, i, k1 + E * k2);
        }
    };
    if constexpr (sizeof(R) >= 8) {
        // FP64 / double-float butterflies are long: one copy of the
        // P-point DFT keeps the kernel inside the instruction cache
#pragma unroll 1
        for (int ii = 0; ii < E / P; ii++) column(ii);
    } else {
#pragma unroll
        for (int ii = 0; ii < E / P; ii++) column(ii);
    }
}

// contiguous lines l (elements l*L + j), p fastest in the CTA
template <typename R, int E, int P, int DIR, class Pro, class Store>
__global__ void __launch_bounds__(FsThreads<R>::value)
k_fs_contig(const cx<R>* __restrict__ in, int64_t nlines, const void* twg, Pro pro, Store store)
{
    using S = FsShape<R, E, P>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R>* tw = reinterpret_cast<cx<R>*>(smem_raw);
    cx<R>* xa = tw + S::L;
    const int t = threadIdx.x;
    const int p = t % P, w = t / P;
    const int64_t l = (int64_t)blockIdx.x * S::W + w;
    const bool act = l < nlines;
    fs_load_tw<R>(tw, twg, S::L);
    cx<R> x[E];
#pragma unroll
    for (int m = 0; m < E; m++) {
        const int j = p + P * m;
        x[m] = act ? pro(in[l * S::L + j], l, 0, j) : mk<R>(0, 0);
    }
    __syncthreads();
    fs_phase1<R, E, P, DIR>(x, p, xa + w * S::LD, tw);
    __syncthreads();
    auto column = [&](int ii) {
        const int k1 = p + P * ii;
        cx<R> u[P];
#pragma unroll
        for (int q = 0; q < P; q++) u[q] = xa[w * S::LD + k1 * S::KS + q];
        dft_reg<P, DIR, S::L, R>(u, tw);
        if (act) {
#pragma unroll
            for (int k2 = 0; k2 < P; k2++) store(u[k2], l, 0, k1 + E * k2);
        }
    };
    if constexpr (sizeof(R) >= 8) {
#pragma unroll 1
        for (int ii = 0; ii < E / P; ii++) column(ii);
    } else {
#pragma unroll
        for (int ii = 0; ii < E / P; ii++) column(ii);
    }
}

// forward real-to-complex rows (2-for-1, see k_r2c_rows): after the
// transform the complex line is staged in natural order (same buffer, after
// a barrier) for the split into the two half spectra.
template <typename R, int E, int P, class Src>
__global__ void __launch_bounds__(FsThreads<R>::value)
k_fs_r2c(Src src, int64_t nrows, cx<R>* __restrict__ out, const void* twg)
{
    using S = FsShape<R, E, P>;
    constexpr int X = S::L, Xh = X / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R>* tw = reinterpret_cast<cx<R>*>(smem_raw);
    cx<R>* xa = tw + S::L;
    const int t = threadIdx.x;
    const int p = t % P, w = t / P;
    const int64_t r0 = (int64_t)blockIdx.x * 2 * S::W;
    const int64_t ra = r0 + 2 * w, rb = ra + 1;
    fs_load_tw<R>(tw, twg, S::L);
    cx<R> x[E];
#pragma unroll
    for (int m = 0; m < E; m++) {
        const int j = p + P * m;
        x[m] = mk<R>(ra < nrows ? src(ra, j) : (R)0, rb < nrows ? src(rb, j) : (R)0);
    }
    __syncthreads();
    fs_phase1<R, E, P, -1>(x, p, xa + w * S::LD, tw);
    __syncthreads();
    // gather this thread's columns, then reuse the buffer in natural order
#pragma unroll
    for (int ii = 0; ii < E / P; ii++)
#pragma unroll
        for (int q = 0; q < P; q++) x[ii * P + q] = xa[w * S::LD + (p + P * ii) * S::KS + q];
    __syncthreads();
#pragma unroll
    for (int ii = 0; ii < E / P; ii++) {
        const int k1 = p + P * ii;
        dft_reg<P, -1, S::L, R>(x + ii * P, tw);
#pragma unroll
        for (int k2 = 0; k2 < P; k2++) xa[w * S::LD + k1 + E * k2] = x[ii * P + k2];
    }
    __syncthreads();
    for (int idx = t; idx < S::W * Xh; idx += blockDim.x) {
        const int ww = idx / Xh, k = idx - ww * Xh;
        const int64_t a = r0 + 2 * ww, b = a + 1;
        const cx<R> zk = xa[ww * S::LD + k];
        const cx<R> zn = xa[ww * S::LD + (k == 0 ? 0 : X - k)];
        const cx<R> A = mk<R>((zk.x + zn.x) * (R)0.5, (zk.y - zn.y) * (R)0.5);
        const cx<R> d = mk<R>(zk.x - zn.x, zk.y + zn.y);
        const cx<R> B = mk<R>(d.y * (R)0.5, -d.x * (R)0.5);
        if (a < nrows) out[a * Xh + k] = A;
        if (b < nrows) out[b * Xh + k] = B;
    }
}

// inverse complex-to-real rows (2-for-1, see k_c2r_rows), batched: the
// component index is the fastest grid index.
template <typename R, int E, int P, class Sink, typename In = cx<R>>
__global__ void __launch_bounds__(FsThreads<R>::value)
k_fs_c2r(const In* __restrict__ in, int64_t nrows, Sink sink, const void* twg, int nbatch)
{
    using S = FsShape<R, E, P>;
    constexpr int X = S::L, Xh = X / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<R>* tw = reinterpret_cast<cx<R>*>(smem_raw);
    cx<R>* xa = tw + S::L;
    const int t = threadIdx.x;
    const int p = t % P, w = t / P;
    const int batch = blockIdx.x % nbatch;
    const int64_t tile = blockIdx.x / nbatch;
    const int64_t ra = tile * 2 * S::W + 2 * w, rb = ra + 1;
    const In* ba = in + ((int64_t)batch * nrows + ra) * Xh;
    const In* bb = ba + Xh;
    const bool va = ra < nrows, vb = rb < nrows;
    fs_load_tw<R>(tw, twg, S::L);
    cx<R> x[E];
#pragma unroll
    for (int m = 0; m < E; m++) {
        const int k = p + P * m;
        const int kk = k < Xh ? k : X - k;
        cx<R> A = va ? load_cx(ba[kk]) : mk<R>(0, 0);
        cx<R> B = vb ? load_cx(bb[kk]) : mk<R>(0, 0);
        if (kk == 0 || 2 * kk == X) { A.y = 0; B.y = 0; }
        // Z(k) = A + iB below X/2, conj A + i conj B above
        x[m] = k < Xh ? mk<R>(A.x - B.y, A.y + B.x) : mk<R>(A.x + B.y, -A.y + B.x);
    }
    __syncthreads();
    fs_phase1<R, E, P, +1>(x, p, xa + w * S::LD, tw);
    __syncthreads();
#pragma unroll
    for (int ii = 0; ii < E / P; ii++) {
        const int k1 = p + P * ii;
        cx<R> u[P];
#pragma unroll
        for (int q = 0; q < P; q++) u[q] = xa[w * S::LD + k1 * S::KS + q];
        dft_reg<P, +1, S::L, R>(u, tw);
#pragma unroll
        for (int k2 = 0; k2 < P; k2++) {
            const int j = k1 + E * k2;
            if (va) sink(batch, ra, j, u[k2].x);
            if (vb) sink(batch, rb, j, u[k2].y);
        }
    }
}

// Fused z pass of the tensorial correlation (see k_zcorr): per component,
// forward four-step of the template column, product with the image
// spectrum in the (k1 + E k2) layout (held in registers for all K), and the
// inverse four-step run backwards to the natural layout.
// TS / TW: storage of the template spectra and of the output (float2, or
// FP16 / BF16 pairs); gmax (or NULL): the image spectrum is multiplied by
// 1 / *gmax as it is loaded, so that scaled products stay in FP16 range.
template <int E, int P, typename TS = float2, typename TW = float2>
__global__ void __launch_bounds__(FsThreads<float>::value, 2)
k_fs_zcorr(const float2* __restrict__ G, const TS* __restrict__ spec, int K, int tzn, int cz, int64_t ncols,
           TW* __restrict__ out, const void* twg, const float* __restrict__ gmax, float oscale)
{
    using S = FsShape<float, E, P>;
    constexpr int Z = S::L;
    constexpr int ZG = Z | 1;  // odd row stride of the image-spectrum tile
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* tw = reinterpret_cast<float2*>(smem_raw);
    float2* xa = tw + S::L;
    const int t = threadIdx.x;
    const int w = t % S::W, p = t / S::W;
    const int64_t c = (int64_t)blockIdx.x * S::W + w;
    const bool act = c < ncols;
    fs_load_tw<float>(tw, twg, S::L);
    // image-spectrum tile, loaded once for all K components (coalesced: the
    // W columns of a row are adjacent)
    float2* gsm = xa + S::W * S::LD;
    const float gs = (gmax && *gmax > 0.f) ? 1.f / *gmax : 1.f;
    for (int idx = t; idx < S::W * Z; idx += blockDim.x) {
        const int z = idx / S::W, ww = idx - z * S::W;
        const int64_t cc = (int64_t)blockIdx.x * S::W + ww;
        gsm[ww * ZG + z] = cc < ncols ? cscale(G[(int64_t)z * ncols + cc], gs) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float2* gl = gsm + w * ZG;
    float2* xl = xa + w * S::LD;
    for (int a = 0; a < K; a++) {
        const TS* sp = spec + (int64_t)a * tzn * ncols;
        float2 x[E];
#pragma unroll
        for (int m = 0; m < E; m++) {
            // template row j lands on z = (j - cz) mod Z
            int j = p + P * m + cz;
            if (j >= Z) j -= Z;
            x[m] = (act && j < tzn) ? load_cx(sp[(int64_t)j * ncols + c]) : make_float2(0.f, 0.f);
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
            for (int k2 = 0; k2 < P; k2++) u[k2] = cmulconj(gl[k1 + E * k2], u[k2]);
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
        __syncthreads();  // all reads of xl done before the next component writes it
    }
}

// ---------------------------------------------------------- dispatchers --

// (E, P) of a length handled by the register kernels, or false
inline bool fs_split(int L, int& E, int& P)
{
    switch (L) {
        case 64: E = 8; P = 8; return true;
        case 128: E = 16; P = 8; return true;
        case 200: E = 20; P = 10; return true;
        case 256: E = 16; P = 16; return true;
        case 512: E = 32; P = 16; return true;
        case 1024: E = 32; P = 32; return true;
        default: return false;
    }
}

#define TTM_FS_SWITCH(L, MACRO)                          \
    switch (L) {                                         \
        case 64: MACRO(8, 8); break;                     \
        case 128: MACRO(16, 8); break;                   \
        case 200: MACRO(20, 10); break;                  \
        case 256: MACRO(16, 16); break;                  \
        case 512: MACRO(32, 16); break;                  \
        case 1024: MACRO(32, 32); break;                 \
        default: throw Error{E_INTERNAL, "no register FFT for this length"}; \
    }

template <typename R, int DIR, class Pro, class Store, typename In = cx<R>>
inline void launch_strided_any(const In* in, StridedAxis ax, const LenPlan& pl, Pro pro, Store store,
                               cudaStream_t st)
{
    if constexpr (std::is_same<R, df64>::value) {
        if (!pl.no_reg && line3_length(pl.L)) {
            launch_line3_strided<DIR>(in, ax, pl, pro, store, st);
            TTM_LAUNCH_CHECK();
            return;
        }
    }
    int E, P;
    if (pl.no_reg || !fs_split(pl.L, E, P)) { launch_strided<R, DIR>(in, ax, pl, pro, store, st); return; }
#define TTM_L(E_, P_)                                                                          \
    {                                                                                          \
        using S = FsShape<R, E_, P_>;                                                          \
        auto k = k_fs_strided<R, E_, P_, DIR, Pro, Store, In>;                                   \
        set_smem(k, S::SMEM);                                                                  \
        int64_t grid = ax.outer * ceil_div(ax.inner, S::W);                                    \
        TTM_REQUIRE(grid < (1ll << 31), E_SHAPE, "strided pass grid too large");               \
        k<<<(unsigned)grid, S::THREADS, S::SMEM, st>>>(in, ax, pl.tw, pro, store);             \
    }
    TTM_FS_SWITCH(pl.L, TTM_L)
#undef TTM_L
    TTM_LAUNCH_CHECK();
}

template <typename R, int DIR, class Pro, class Store>
inline void launch_contig_any(const cx<R>* in, int64_t nlines, const LenPlan& pl, Pro pro, Store store,
                              cudaStream_t st)
{
    if constexpr (std::is_same<R, df64>::value) {
        if (!pl.no_reg && line3_length(pl.L)) {
            launch_line3_contig<DIR>(in, nlines, pl, pro, store, st);
            TTM_LAUNCH_CHECK();
            return;
        }
    }
    int E, P;
    if (pl.no_reg || !fs_split(pl.L, E, P)) { launch_contig<R, DIR>(in, nlines, pl, pro, store, st); return; }
#define TTM_L(E_, P_)                                                                          \
    {                                                                                          \
        using S = FsShape<R, E_, P_>;                                                          \
        auto k = k_fs_contig<R, E_, P_, DIR, Pro, Store>;                                      \
        set_smem(k, S::SMEM);                                                                  \
        k<<<(unsigned)ceil_div(nlines, S::W), S::THREADS, S::SMEM, st>>>(in, nlines, pl.tw, pro, store); \
    }
    TTM_FS_SWITCH(pl.L, TTM_L)
#undef TTM_L
    TTM_LAUNCH_CHECK();
}

template <typename R, class Src>
inline void launch_r2c_any(Src src, int64_t nrows, cx<R>* out, const LenPlan& pl, cudaStream_t st)
{
    int E, P;
    if (pl.no_reg || !fs_split(pl.L, E, P)) { launch_r2c_rows<R>(src, nrows, out, pl, st); return; }
#define TTM_L(E_, P_)                                                                          \
    {                                                                                          \
        using S = FsShape<R, E_, P_>;                                                          \
        auto k = k_fs_r2c<R, E_, P_, Src>;                                                     \
        set_smem(k, S::SMEM);                                                                  \
        k<<<(unsigned)ceil_div(nrows, 2 * S::W), S::THREADS, S::SMEM, st>>>(src, nrows, out, pl.tw); \
    }
    TTM_FS_SWITCH(pl.L, TTM_L)
#undef TTM_L
    TTM_LAUNCH_CHECK();
}

template <typename TS, typename TW>
inline bool launch_zcorr_fs(const float2* G, const TS* spec, int K, int tzn, int cz, int64_t ncols, TW* out,
                            const LenPlan& pz, const float* gmax, float oscale, cudaStream_t st)
{
    int E, P;
    if (pz.no_reg || !fs_split(pz.L, E, P)) return false;
#define TTM_L(E_, P_)                                                                          \
    {                                                                                          \
        using S = FsShape<float, E_, P_>;                                                      \
        const size_t smem = S::SMEM + (size_t)S::W * (S::L | 1) * sizeof(float2);              \
        auto k = k_fs_zcorr<E_, P_, TS, TW>;                                                   \
        set_smem(k, smem);                                                                     \
        k<<<(unsigned)ceil_div(ncols, S::W), S::THREADS, smem, st>>>(G, spec, K, tzn, cz, ncols, out, pz.tw, gmax, oscale); \
    }
    TTM_FS_SWITCH(pz.L, TTM_L)
#undef TTM_L
    TTM_LAUNCH_CHECK();
    return true;
}

template <typename R, class Sink, typename In = cx<R>>
inline void launch_c2r_any(const In* in, int64_t nrows, Sink sink, const LenPlan& pl, int nbatch,
                           cudaStream_t st)
{
    int E, P;
    if (pl.no_reg || !fs_split(pl.L, E, P)) { launch_c2r_rows<R>(in, nrows, sink, pl, nbatch, st); return; }
#define TTM_L(E_, P_)                                                                          \
    {                                                                                          \
        using S = FsShape<R, E_, P_>;                                                          \
        auto k = k_fs_c2r<R, E_, P_, Sink, In>;                                                 \
        set_smem(k, S::SMEM);                                                                  \
        int64_t grid = ceil_div(nrows, 2 * S::W) * nbatch;                                     \
        TTM_REQUIRE(grid < (1ll << 31), E_SHAPE, "c2r pass grid too large");                   \
        k<<<(unsigned)grid, S::THREADS, S::SMEM, st>>>(in, nrows, sink, pl.tw, nbatch);        \
    }
    TTM_FS_SWITCH(pl.L, TTM_L)
#undef TTM_L
    TTM_LAUNCH_CHECK();
}

}  // namespace ttm
