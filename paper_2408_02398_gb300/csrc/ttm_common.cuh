// ttm_common.cuh -- shared device/host helpers of the TTM CUDA library.
//
// Complex numbers are float2 / double2 (x = real, y = imaginary) so that a
// complex element moves with one 8- or 16-byte vector access. Volumes are
// C-order [Z][Y][X] with x fastest; half spectra of real volumes are
// [Z][Y][X/2+1].
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

namespace ttm {

template <typename R> struct cx_of;
template <> struct cx_of<float> { using type = float2; };
template <> struct cx_of<double> { using type = double2; };
template <typename R> using cx = typename cx_of<R>::type;

template <typename R> __host__ __device__ __forceinline__ cx<R> mk(R a, R b) { cx<R> c; c.x = a; c.y = b; return c; }
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b)
{
    C c;
    c.x = a.x * b.x - a.y * b.y;
    c.y = a.x * b.y + a.y * b.x;
    return c;
}
// a * conj(b)
template <typename C> __host__ __device__ __forceinline__ C cmulconj(C a, C b)
{
    C c;
    c.x = a.x * b.x + a.y * b.y;
    c.y = a.y * b.x - a.x * b.y;
    return c;
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) { a.x *= s; a.y *= s; return a; }
// multiply by DIR * i (DIR = -1 forward, +1 inverse)
template <int DIR, typename C> __device__ __forceinline__ C cmul_diri(C a)
{
    C c;
    if (DIR > 0) { c.x = -a.y; c.y = a.x; }
    else { c.x = a.y; c.y = -a.x; }
    return c;
}

// status codes mirrored from include/ttm.h (kept in sync by a static test)
enum Status { OK = 0, E_INVALID_ARG = 1, E_SHAPE = 2, E_UNSUPPORTED = 3, E_OOM = 4, E_CUDA = 5,
              E_TIMEOUT = 6, E_INTERNAL = 7 };

struct Error {
    int code;
    std::string msg;
};

#define TTM_CUDA_TRY(expr)                                                                       \
    do {                                                                                         \
        cudaError_t e__ = (expr);                                                                \
        if (e__ != cudaSuccess)                                                                  \
            throw ::ttm::Error{::ttm::E_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e__)}; \
    } while (0)

#define TTM_REQUIRE(cond, code, text)                                                            \
    do {                                                                                         \
        if (!(cond)) throw ::ttm::Error{(code), (text)};                                         \
    } while (0)

// every kernel launch is followed by this check, which also counts it
void count_launch();
#define TTM_LAUNCH_CHECK()                  \
    do {                                    \
        ::ttm::count_launch();              \
        TTM_CUDA_TRY(cudaGetLastError());   \
    } while (0)

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Index on a template axis (length t, centre t/2) of the offset p that is
// stored at grid index i of a wrapped axis of length n >= t (p = i or
// p = i - n), or -1 if no template offset lands there.
__device__ __forceinline__ int wrap_to_template(int i, int n, int t)
{
    int q = i + t / 2;          // p = i >= 0
    if (q < t) return q;
    q = i - n + t / 2;          // p = i - n < 0
    return q >= 0 ? q : -1;
}


}  // namespace ttm
