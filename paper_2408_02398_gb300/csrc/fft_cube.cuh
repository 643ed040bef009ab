// fft_cube.cuh -- double-float FFT passes for lines of length L = R^3
// (R = 8: L = 512) held in registers.
//
// With j = p + R^2 m and k = k1 + R s + R^2 t (p < R^2; m, k1, s, t < R),
// and p = q + R r (q, r < R) inside the length-R^2 transform:
//   a[p][k1]            = w_L^{p k1}    sum_m x[p + R^2 m] w_R^{m k1}
//   c[k1][q][s]         = w_{R^2}^{q s} sum_r a[q + R r][k1] w_R^{r s}
//   X[k1 + R s + R^2 t] =               sum_q c[k1][q][s] w_R^{q t}
// (w_n = exp(-2 pi i / n), conjugated for the inverse). A line has R^2
// threads; each holds R values, does one R-point DFT per level in
// registers, and two shared-memory exchanges hand it the next level's
// inputs. Thread u of a line plays p = u at the first level, (q, k1) =
// (u mod R, u / R) at the second and (k1, s) = (u mod R, u / R) at the
// third, so the loads x[u + R^2 m] and the stores X[u + R^2 t] are both
// unit-stride in u.
//
// Exchange layout (16-byte elements, one line): a[p][k1] at k1 KS + p and
// c[k1][q][s] at k1 KS + s RS + q, with RS = R + 1 and KS = R RS + 1, so
// that every group of 8 threads served by one shared-memory wavefront
// touches 8 distinct 16-byte bank groups at each of the four accesses;
// the line stride LW spreads the NL lines that share such a group.
#pragma once

#include "fft.cuh"

namespace ttm {

template <int R, int NL> struct CubeShape {
    static constexpr int L = R * R * R;
    static constexpr int T = R * R;                       // threads per line
    static constexpr int RS = R + 1;                      // stride of the s rows of exchange 2
    static constexpr int KS = R * RS + 1;                 // stride of the k1 rows
    static constexpr int LW = R * KS + (NL >= 8 ? 1 : 8 / NL);  // line stride
    static constexpr int NTW1 = (R - 1) * T;              // first-level twiddles [k1 - 1][p]
    static constexpr int NTW2 = (R - 1) * R;              // second-level twiddles [s - 1][q]
    static constexpr int THREADS = NL * T;
    static constexpr size_t SMEM = ((size_t)NL * LW + NTW1 + NTW2) * sizeof(dcx);
};

// the two twiddle tables of a CTA from the global table exp(-2 pi i t / L)
template <int R, int NL, int DIR>
__device__ __forceinline__ void cube_twiddles(dcx* tw1, dcx* tw2, const void* twg)
{
    using S = CubeShape<R, NL>;
    const dcx* g = reinterpret_cast<const dcx*>(twg);
    for (int i = threadIdx.x; i < S::NTW1 + S::NTW2; i += blockDim.x) {
        int t;
        if (i < S::NTW1) t = (i % S::T) * (i / S::T + 1);                     // p k1
        else t = R * ((i - S::NTW1) % R) * ((i - S::NTW1) / R + 1);           // R q s
        dcx w = g[t];
        if (DIR > 0) w.y = -w.y;
        if (i < S::NTW1) tw1[i] = w;
        else tw2[i - S::NTW1] = w;
    }
}

// the transform of one line: x holds x[u + R^2 m] on entry and
// X[u + R^2 t] on return; xb is the line's exchange buffer. Contains three
// __syncthreads (every thread of the CTA must call it).
template <int R, int NL, int DIR>
__device__ __forceinline__ void cube_fft(dcx* x, int u, dcx* xb, const dcx* tw1, const dcx* tw2)
{
    using S = CubeShape<R, NL>;
    dft<R, DIR, df64>(x);
#pragma unroll
    for (int k1 = 1; k1 < R; k1++) x[k1] = cmul(x[k1], tw1[(k1 - 1) * S::T + u]);
#pragma unroll
    for (int k1 = 0; k1 < R; k1++) xb[k1 * S::KS + u] = x[k1];
    __syncthreads();
    {
        const int q = u % R, k1 = u / R;
#pragma unroll
        for (int r = 0; r < R; r++) x[r] = xb[k1 * S::KS + q + R * r];
        dft<R, DIR, df64>(x);
#pragma unroll
        for (int s = 1; s < R; s++) x[s] = cmul(x[s], tw2[(s - 1) * R + q]);
        __syncthreads();
#pragma unroll
        for (int s = 0; s < R; s++) xb[k1 * S::KS + s * S::RS + q] = x[s];
    }
    __syncthreads();
    {
        const int k1 = u % R, s = u / R;
#pragma unroll
        for (int q = 0; q < R; q++) x[q] = xb[k1 * S::KS + s * S::RS + q];
        dft<R, DIR, df64>(x);
    }
}

// contiguous lines: line l has elements l L + j; NL lines per CTA, thread
// u + T w works on line w (functors get (o = l, i = 0, j))
template <int R, int NL, int DIR, class Pro, class Store>
__global__ void __launch_bounds__(CubeShape<R, NL>::THREADS)
k_cube_contig(const dcx* __restrict__ in, int64_t nlines, const void* twg, Pro pro, Store store)
{
    using S = CubeShape<R, NL>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    dcx* xb = reinterpret_cast<dcx*>(smem_raw);
    dcx* tw1 = xb + NL * S::LW;
    dcx* tw2 = tw1 + S::NTW1;
    cube_twiddles<R, NL, DIR>(tw1, tw2, twg);
    const int u = threadIdx.x % S::T, w = threadIdx.x / S::T;
    const int64_t l = (int64_t)blockIdx.x * NL + w;
    const bool act = l < nlines;
    dcx x[R];
#pragma unroll
    for (int m = 0; m < R; m++) {
        const int j = u + S::T * m;
        x[m] = act ? pro(in[l * S::L + j], l, 0, j) : mk<df64>(df64(0.f, 0.f), df64(0.f, 0.f));
    }
    __syncthreads();
    cube_fft<R, NL, DIR>(x, u, xb + w * S::LW, tw1, tw2);
    if (act) {
#pragma unroll
        for (int t = 0; t < R; t++) store(x[t], l, 0, u + S::T * t);
    }
}

// strided axis: lines (o, i) with elements o os + i + j s; NL lines adjacent
// in i per CTA, thread w + NL u works on line i0 + w (w fastest, so a warp
// reads runs of NL adjacent elements)
template <int R, int NL, int DIR, class Pro, class Store, typename In>
__global__ void __launch_bounds__(CubeShape<R, NL>::THREADS)
k_cube_strided(const In* __restrict__ in, StridedAxis ax, const void* twg, Pro pro, Store store)
{
    using S = CubeShape<R, NL>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    dcx* xb = reinterpret_cast<dcx*>(smem_raw);
    dcx* tw1 = xb + NL * S::LW;
    dcx* tw2 = tw1 + S::NTW1;
    cube_twiddles<R, NL, DIR>(tw1, tw2, twg);
    const int w = threadIdx.x % NL, u = threadIdx.x / NL;
    const int64_t tiles = (ax.inner + NL - 1) / NL;
    const int64_t o = blockIdx.x / tiles;
    const int64_t i = (blockIdx.x - o * tiles) * NL + w;
    const bool act = i < ax.inner;
    const In* src = in + o * ax.os + i;
    dcx x[R];
#pragma unroll
    for (int m = 0; m < R; m++) {
        const int j = u + S::T * m;
        x[m] = act ? pro(load_cx(src[(int64_t)j * ax.s]), o, i, j) : mk<df64>(df64(0.f, 0.f), df64(0.f, 0.f));
    }
    __syncthreads();
    cube_fft<R, NL, DIR>(x, u, xb + w * S::LW, tw1, tw2);
    if (act) {
#pragma unroll
        for (int t = 0; t < R; t++) store(x[t], o, i, u + S::T * t);
    }
}

// lengths these passes serve
__host__ __device__ constexpr bool cube_length(int L) { return L == 512; }

template <int DIR, class Pro, class Store>
inline void launch_cube_contig(const dcx* in, int64_t nlines, const LenPlan& pl, Pro pro, Store store,
                               cudaStream_t st)
{
    constexpr int R = 8, NL = 4;
    using S = CubeShape<R, NL>;
    auto k = k_cube_contig<R, NL, DIR, Pro, Store>;
    set_smem(k, S::SMEM);
    const int64_t grid = ceil_div(nlines, (int64_t)NL);
    TTM_REQUIRE(grid < (1ll << 31), E_SHAPE, "contiguous pass grid too large");
    k<<<(unsigned)grid, S::THREADS, S::SMEM, st>>>(in, nlines, pl.tw, pro, store);
}

template <int DIR, class Pro, class Store, typename In>
inline void launch_cube_strided(const In* in, StridedAxis ax, const LenPlan& pl, Pro pro, Store store,
                                cudaStream_t st)
{
    constexpr int R = 8, NL = 4;
    using S = CubeShape<R, NL>;
    auto k = k_cube_strided<R, NL, DIR, Pro, Store, In>;
    set_smem(k, S::SMEM);
    const int64_t grid = ax.outer * ceil_div(ax.inner, (int64_t)NL);
    TTM_REQUIRE(grid < (1ll << 31), E_SHAPE, "strided pass grid too large");
    k<<<(unsigned)grid, S::THREADS, S::SMEM, st>>>(in, ax, pl.tw, pro, store);
}

}  // namespace ttm
