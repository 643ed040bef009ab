// fft_line3.cuh -- double-float FFT passes whose lines are held in
// registers, for lengths L = R1 R2 R3 with radices in {2, 3, 4, 5, 7, 8}.
//
// With j = p + P m and k = k1 + R1 s + R1 R2 t (P = R2 R3; p < P; m, k1 <
// R1; s < R2; t < R3), and p = q + R3 r (q < R3, r < R2) inside the
// length-P transform:
//   a[p][k1]                = w_L^{p k1}  sum_m x[p + P m] w_R1^{m k1}
//   c[k1][q][s]             = w_P^{q s}   sum_r a[q + R3 r][k1] w_R2^{r s}
//   X[k1 + R1 s + R1 R2 t]  =             sum_q c[k1][q][s] w_R3^{q t}
// (w_n = exp(-2 pi i / n), conjugated for the inverse). Each level is one
// R-point DFT per thread in registers; two shared-memory exchanges hand a
// thread the next level's inputs. Thread u of a line plays p = u at the
// first level (u < P), (q, k1) = (u mod R3, u / R3) at the second
// (u < R1 R3) and (k1, s) = (u mod R1, u / R1) at the third (u < R1 R2),
// so it loads x[u + P m] and ends holding X[u + R1 R2 t]: both unit-stride
// in u. The transform with the radices reversed, (R3, R2, R1), takes its
// input in exactly that layout, so a forward transform, a pointwise
// product and an inverse transform chain with no further exchange.
//
// Exchange layout (16-byte elements, one line): a[p][k1] at k1 KS + p,
// c[k1][q][s] at k1 KS + s RS + q, RS = R3 + 1 and KS = 1 mod 8. For
// 8 x 8 x 8 every group of 8 consecutive threads (one shared-memory
// wavefront of 16-byte accesses) then meets 8 distinct bank groups at each
// exchange; where 8 lines sit side by side in a wavefront (NL = 8, w
// fastest) an odd line stride alone makes every access conflict-free.
#pragma once

#include "fft.cuh"

namespace ttm {

__host__ __device__ constexpr int l3_max(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int l3_round1(int n) { return n + ((9 - (n & 7)) & 7); }  // smallest >= n, = 1 mod 8

template <int R1, int R2, int R3> struct Line3 {
    static constexpr int L = R1 * R2 * R3;
    static constexpr int P = R2 * R3;                              // threads of level 1
    static constexpr int T = l3_max(P, l3_max(R1 * R3, R1 * R2));  // threads per line
    static constexpr int RMAX = l3_max(R1, l3_max(R2, R3));
    static constexpr int RS = R3 + 1;
    static constexpr int KS = l3_round1(l3_max(P, (R2 - 1) * RS + R3));
    static constexpr int ROWS = R1 * KS;                           // exchange entries of a line
    static constexpr int NTW1 = (R1 - 1) * P;                      // level-1 twiddles [k1 - 1][p]
    static constexpr int NTW2 = (R2 - 1) * R3;                     // level-2 twiddles [s - 1][q]
    static constexpr int NTW = NTW1 + NTW2;
};

// the twiddles of Line3<R1, R2, R3> in direction DIR from the global table
// exp(-2 pi i t / L): tw[(k1 - 1) P + p] = w^{p k1}, then
// tw[NTW1 + (s - 1) R3 + q] = w^{R1 q s}
template <int R1, int R2, int R3, int DIR>
__device__ __forceinline__ void line3_twiddles(dcx* tw, const void* twg)
{
    using S = Line3<R1, R2, R3>;
    const dcx* g = reinterpret_cast<const dcx*>(twg);
    for (int i = threadIdx.x; i < S::NTW; i += blockDim.x) {
        const int t = i < S::NTW1 ? (i % S::P) * (i / S::P + 1)
                                  : R1 * ((i - S::NTW1) % R3) * ((i - S::NTW1) / R3 + 1);
        dcx w = g[t];
        if (DIR > 0) w.y = -w.y;
        tw[i] = w;
    }
}

// one transform of the line whose exchange buffer is xb: thread u holds
// x[u + P m] (m < R1) on entry if u < P, and X[u + R1 R2 t] (t < R3) on
// return if u < R1 R2. Every thread of the CTA calls it (four barriers;
// the first one orders it after whatever used xb or the twiddles before).
template <int R1, int R2, int R3, int DIR>
__device__ __forceinline__ void line3_run(dcx* x, int u, dcx* xb, const dcx* tw)
{
    using S = Line3<R1, R2, R3>;
    __syncthreads();
    if (u < S::P) {
        dft<R1, DIR, df64>(x);
#pragma unroll
        for (int k1 = 1; k1 < R1; k1++) x[k1] = cmul(x[k1], tw[(k1 - 1) * S::P + u]);
#pragma unroll
        for (int k1 = 0; k1 < R1; k1++) xb[k1 * S::KS + u] = x[k1];
    }
    __syncthreads();
    const int q = u % R3, k1b = u / R3;
    const bool act2 = u < R1 * R3;
    if (act2) {
#pragma unroll
        for (int r = 0; r < R2; r++) x[r] = xb[k1b * S::KS + q + R3 * r];
        dft<R2, DIR, df64>(x);
#pragma unroll
        for (int s = 1; s < R2; s++) x[s] = cmul(x[s], tw[S::NTW1 + (s - 1) * R3 + q]);
    }
    __syncthreads();
    if (act2) {
#pragma unroll
        for (int s = 0; s < R2; s++) xb[k1b * S::KS + s * S::RS + q] = x[s];
    }
    __syncthreads();
    if (u < R1 * R2) {
        const int k1 = u % R1, s = u / R1;
#pragma unroll
        for (int qq = 0; qq < R3; qq++) x[qq] = xb[k1 * S::KS + s * S::RS + qq];
        dft<R3, DIR, df64>(x);
    }
}

__device__ __forceinline__ dcx dcx_zero() { return mk<df64>(df64(0.f, 0.f), df64(0.f, 0.f)); }

// line stride of NL lines: 8 / NL mod 8 (NL < 8) or 1 mod 8 (NL >= 8), so
// that the NL lines sharing a wavefront fall on distinct bank groups
__host__ __device__ constexpr int l3_line_stride(int rows, int NL)
{
    return rows + ((((NL >= 8 ? 1 : 8 / NL) - rows) % 8 + 8) % 8);
}

// contiguous lines: line l has elements l L + j; NL lines per CTA, thread
// u + T w works on line w (functors get (o = l, i = 0, j))
template <int R1, int R2, int R3, int NL, int DIR, class Pro, class Store>
__global__ void __launch_bounds__(NL * Line3<R1, R2, R3>::T, 65536 / (NL * Line3<R1, R2, R3>::T * 64))
k_line3_contig(const dcx* __restrict__ in, int64_t nlines, const void* twg, Pro pro, Store store)
{
    using S = Line3<R1, R2, R3>;
    constexpr int LW = l3_line_stride(S::ROWS, NL);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    dcx* tw = reinterpret_cast<dcx*>(smem_raw);
    dcx* xb = tw + S::NTW;
    line3_twiddles<R1, R2, R3, DIR>(tw, twg);
    const int u = threadIdx.x % S::T, w = threadIdx.x / S::T;
    const int64_t l = (int64_t)blockIdx.x * NL + w;
    const bool act = l < nlines;
    dcx x[S::RMAX];
    if (u < S::P) {
#pragma unroll
        for (int m = 0; m < R1; m++) {
            const int j = u + S::P * m;
            x[m] = act ? pro(in[l * S::L + j], l, 0, j) : dcx_zero();
        }
    }
    line3_run<R1, R2, R3, DIR>(x, u, xb + w * LW, tw);
    if (act && u < R1 * R2) {
#pragma unroll
        for (int t = 0; t < R3; t++) store(x[t], l, 0, u + R1 * R2 * t);
    }
}

// contiguous lines produced by a source functor: src(l, j) gives element j
// of line l (so the line can be formed from other data as it is loaded)
template <int R1, int R2, int R3, int NL, int DIR, class Src, class Store>
__global__ void __launch_bounds__(NL * Line3<R1, R2, R3>::T, 65536 / (NL * Line3<R1, R2, R3>::T * 64))
k_line3_contig_src(int64_t nlines, const void* twg, Src src, Store store)
{
    using S = Line3<R1, R2, R3>;
    constexpr int LW = l3_line_stride(S::ROWS, NL);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    dcx* tw = reinterpret_cast<dcx*>(smem_raw);
    dcx* xb = tw + S::NTW;
    line3_twiddles<R1, R2, R3, DIR>(tw, twg);
    const int u = threadIdx.x % S::T, w = threadIdx.x / S::T;
    const int64_t l = (int64_t)blockIdx.x * NL + w;
    const bool act = l < nlines;
    dcx x[S::RMAX];
    if (u < S::P) {
#pragma unroll
        for (int m = 0; m < R1; m++) x[m] = act ? src(l, u + S::P * m) : dcx_zero();
    }
    line3_run<R1, R2, R3, DIR>(x, u, xb + w * LW, tw);
    if (act && u < R1 * R2) {
#pragma unroll
        for (int t = 0; t < R3; t++) store(x[t], l, 0, u + R1 * R2 * t);
    }
}

// strided axis: lines (o, i) with elements o os + i + j s; NL lines adjacent
// in i per CTA, thread w + NL u works on line i0 + w (w fastest, so a warp
// reads runs of NL adjacent elements)
template <int R1, int R2, int R3, int NL, int DIR, class Pro, class Store, typename In>
__global__ void __launch_bounds__(NL * Line3<R1, R2, R3>::T, 65536 / (NL * Line3<R1, R2, R3>::T * 64))
k_line3_strided(const In* __restrict__ in, StridedAxis ax, const void* twg, Pro pro, Store store)
{
    using S = Line3<R1, R2, R3>;
    constexpr int LW = l3_line_stride(S::ROWS, NL);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    dcx* tw = reinterpret_cast<dcx*>(smem_raw);
    dcx* xb = tw + S::NTW;
    line3_twiddles<R1, R2, R3, DIR>(tw, twg);
    const int w = threadIdx.x % NL, u = threadIdx.x / NL;
    const int64_t tiles = (ax.inner + NL - 1) / NL;
    const int64_t o = blockIdx.x / tiles;
    const int64_t i = (blockIdx.x - o * tiles) * NL + w;
    const bool act = i < ax.inner;
    const In* src = in + o * ax.os + i;
    dcx x[S::RMAX];
    if (u < S::P) {
#pragma unroll
        for (int m = 0; m < R1; m++) {
            const int j = u + S::P * m;
            x[m] = act ? pro(load_cx(src[(int64_t)j * ax.s]), o, i, j) : dcx_zero();
        }
    }
    line3_run<R1, R2, R3, DIR>(x, u, xb + w * LW, tw);
    if (act && u < R1 * R2) {
#pragma unroll
        for (int t = 0; t < R3; t++) store(x[t], o, i, u + R1 * R2 * t);
    }
}

// Fused z pass of the local sums with the lines in registers: per group of
// NL adjacent (y, x) columns of zd (ncols of them, z stride ncols), the
// forward transform along z (R1 R2 R3), the product with the mask spectrum
// (mask(v, 0, column, kz)) and the inverse transform (R3 R2 R1), in place.
template <int R1, int R2, int R3, int NL, class Mask>
__global__ void __launch_bounds__(NL * Line3<R1, R2, R3>::T, 65536 / (NL * Line3<R1, R2, R3>::T * 64))
k_line3_zmask(dcx* __restrict__ zd, int64_t ncols, const void* twg, Mask mask)
{
    using F = Line3<R1, R2, R3>;
    using B = Line3<R3, R2, R1>;
    static_assert(F::T == B::T, "forward and inverse thread counts differ");
    constexpr int LW = l3_line_stride(l3_max(F::ROWS, B::ROWS), NL);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    dcx* twf = reinterpret_cast<dcx*>(smem_raw);
    dcx* twb = twf + F::NTW;
    dcx* xb = twb + B::NTW;
    line3_twiddles<R1, R2, R3, -1>(twf, twg);
    line3_twiddles<R3, R2, R1, +1>(twb, twg);
    const int w = threadIdx.x % NL, u = threadIdx.x / NL;
    const int64_t c = (int64_t)blockIdx.x * NL + w;
    const bool act = c < ncols;
    dcx x[F::RMAX];
    if (u < F::P) {
#pragma unroll
        for (int m = 0; m < R1; m++) x[m] = act ? zd[(int64_t)(u + F::P * m) * ncols + c] : dcx_zero();
    }
    line3_run<R1, R2, R3, -1>(x, u, xb + w * LW, twf);
    if (u < R1 * R2) {
#pragma unroll
        for (int t = 0; t < R3; t++) x[t] = mask(x[t], 0, c, u + R1 * R2 * t);
    }
    line3_run<R3, R2, R1, +1>(x, u, xb + w * LW, twb);
    if (act && u < R3 * R2) {
#pragma unroll
        for (int t = 0; t < R1; t++) zd[(int64_t)(u + R3 * R2 * t) * ncols + c] = x[t];
    }
}

// --------------------------------------------------------------- host --

// lengths served, with their radices (first level first)
#define TTM_LINE3_SWITCH(L, MACRO)                  \
    switch (L) {                                    \
        case 512: MACRO(8, 8, 8); break;            \
        case 256: MACRO(8, 8, 4); break;            \
        case 200: MACRO(8, 5, 5); break;            \
        case 128: MACRO(8, 4, 4); break;            \
        default: throw Error{E_INTERNAL, "no three-level register FFT for this length"}; \
    }
inline bool line3_length(int L) { return L == 512 || L == 256 || L == 200 || L == 128; }

template <int R1, int R2, int R3, int NL>
constexpr size_t line3_smem()
{
    using S = Line3<R1, R2, R3>;
    return ((size_t)S::NTW + (size_t)NL * l3_line_stride(S::ROWS, NL)) * sizeof(dcx);
}

template <int DIR, class Pro, class Store>
inline void launch_line3_contig(const dcx* in, int64_t nlines, const LenPlan& pl, Pro pro, Store store,
                                cudaStream_t st)
{
    const int64_t grid0 = nlines;
#define TTM_L3(R1_, R2_, R3_)                                                                  \
    {                                                                                          \
        constexpr int NL = 4;                                                                  \
        auto k = k_line3_contig<R1_, R2_, R3_, NL, DIR, Pro, Store>;                            \
        constexpr size_t smem = line3_smem<R1_, R2_, R3_, NL>();                               \
        set_smem(k, smem);                                                                     \
        const int64_t grid = ceil_div(grid0, (int64_t)NL);                                     \
        TTM_REQUIRE(grid < (1ll << 31), E_SHAPE, "contiguous pass grid too large");            \
        k<<<(unsigned)grid, NL * Line3<R1_, R2_, R3_>::T, smem, st>>>(in, nlines, pl.tw, pro, store); \
    }
    TTM_LINE3_SWITCH(pl.L, TTM_L3)
#undef TTM_L3
}

template <int DIR, class Src, class Store>
inline void launch_line3_contig_src(int64_t nlines, const LenPlan& pl, Src src, Store store, cudaStream_t st)
{
#define TTM_L3(R1_, R2_, R3_)                                                                  \
    {                                                                                          \
        constexpr int NL = 4;                                                                  \
        auto k = k_line3_contig_src<R1_, R2_, R3_, NL, DIR, Src, Store>;                        \
        constexpr size_t smem = line3_smem<R1_, R2_, R3_, NL>();                               \
        set_smem(k, smem);                                                                     \
        const int64_t grid = ceil_div(nlines, (int64_t)NL);                                    \
        TTM_REQUIRE(grid < (1ll << 31), E_SHAPE, "contiguous pass grid too large");            \
        k<<<(unsigned)grid, NL * Line3<R1_, R2_, R3_>::T, smem, st>>>(nlines, pl.tw, src, store); \
    }
    TTM_LINE3_SWITCH(pl.L, TTM_L3)
#undef TTM_L3
}

template <int DIR, class Pro, class Store, typename In>
inline void launch_line3_strided(const In* in, StridedAxis ax, const LenPlan& pl, Pro pro, Store store,
                                 cudaStream_t st)
{
#define TTM_L3(R1_, R2_, R3_)                                                                  \
    {                                                                                          \
        constexpr int NL = 4;                                                                  \
        auto k = k_line3_strided<R1_, R2_, R3_, NL, DIR, Pro, Store, In>;                       \
        constexpr size_t smem = line3_smem<R1_, R2_, R3_, NL>();                               \
        set_smem(k, smem);                                                                     \
        const int64_t grid = ax.outer * ceil_div(ax.inner, (int64_t)NL);                       \
        TTM_REQUIRE(grid < (1ll << 31), E_SHAPE, "strided pass grid too large");               \
        k<<<(unsigned)grid, NL * Line3<R1_, R2_, R3_>::T, smem, st>>>(in, ax, pl.tw, pro, store); \
    }
    TTM_LINE3_SWITCH(pl.L, TTM_L3)
#undef TTM_L3
}

template <class Mask>
inline void launch_line3_zmask(dcx* zd, int64_t ncols, const LenPlan& pl, Mask mask, cudaStream_t st)
{
#define TTM_L3(R1_, R2_, R3_)                                                                  \
    {                                                                                          \
        constexpr int NL = 8;                                                                  \
        using F = Line3<R1_, R2_, R3_>;                                                        \
        using B = Line3<R3_, R2_, R1_>;                                                        \
        auto k = k_line3_zmask<R1_, R2_, R3_, NL, Mask>;                                        \
        constexpr size_t smem =                                                                \
            ((size_t)F::NTW + B::NTW + (size_t)NL * l3_line_stride(l3_max(F::ROWS, B::ROWS), NL)) * sizeof(dcx); \
        set_smem(k, smem);                                                                     \
        const int64_t grid = ceil_div(ncols, (int64_t)NL);                                     \
        TTM_REQUIRE(grid < (1ll << 31), E_SHAPE, "z pass grid too large");                     \
        k<<<(unsigned)grid, NL * F::T, smem, st>>>(zd, ncols, pl.tw, mask);                    \
    }
    TTM_LINE3_SWITCH(pl.L, TTM_L3)
#undef TTM_L3
}

}  // namespace ttm
