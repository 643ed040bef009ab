// ttm_peaks.cu -- Find Peaks (Sec. 3.4): local maxima of a score map inside
// the valid box, then the P highest with a minimum exclusion distance.
// The device marks the 26-neighbour maxima (ties go to the lower linear
// index) and compacts them; the host orders the candidates by (value desc,
// index asc) and accepts greedily.
#include <algorithm>
#include <string>
#include <vector>

#include "ttm_internal.h"

namespace ttm {

__global__ void k_localmax(const float* __restrict__ s, int Z, int Y, int X, int z0, int z1, int y0, int y1, int x0,
                           int x1, int64_t cap, int64_t* __restrict__ idx, float* __restrict__ val,
                           unsigned long long* __restrict__ count)
{
    const int bx = x1 - x0, by = y1 - y0, bz = z1 - z0;
    const int64_t n = (int64_t)bx * by * bz;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        int x = x0 + (int)(t % bx);
        int64_t r = t / bx;
        int y = y0 + (int)(r % by), z = z0 + (int)(r / by);
        int64_t i = ((int64_t)z * Y + y) * X + x;
        float v = s[i];
        if (!(v == v)) continue;  // NaN is never a peak
        bool is_max = true;
        for (int dz = -1; dz <= 1 && is_max; dz++)
            for (int dy = -1; dy <= 1 && is_max; dy++)
                for (int dx = -1; dx <= 1 && is_max; dx++) {
                    if (!dz && !dy && !dx) continue;
                    int zz = z + dz, yy = y + dy, xx = x + dx;
                    if (zz < z0 || zz >= z1 || yy < y0 || yy >= y1 || xx < x0 || xx >= x1) continue;
                    int64_t j = ((int64_t)zz * Y + yy) * X + xx;
                    float o = s[j];
                    if (o > v || (o == v && j < i)) is_max = false;
                }
        if (!is_max) continue;
        unsigned long long pos = atomicAdd(count, 1ull);
        if ((int64_t)pos < cap) { idx[pos] = i; val[pos] = v; }
    }
}

int find_peaks_run(ttm_plan* P, const float* d_map, int Pk, double min_dist, int64_t* h_idx, float* h_val,
                   cudaStream_t st)
{
    const Prep& p = P->prep;
    int b[6];
    ttm_plan_valid_box(P, b);
    int64_t* cidx = P->cand.as<int64_t>();
    float* cval = reinterpret_cast<float*>(cidx + P->cand_cap);
    unsigned long long* cnt = P->cand_count.as<unsigned long long>();
    TTM_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
    k_localmax<<<32 * P->ctx->num_sms, 256, 0, st>>>(d_map, p.Z, p.Y, p.X, b[0], b[1], b[2], b[3], b[4], b[5], P->cand_cap,
                                           cidx, cval, cnt);
    TTM_LAUNCH_CHECK();
    unsigned long long n = 0;
    TTM_CUDA_TRY(cudaMemcpyAsync(&n, cnt, sizeof(n), cudaMemcpyDeviceToHost, st));
    TTM_CUDA_TRY(cudaStreamSynchronize(st));
    TTM_REQUIRE((int64_t)n <= P->cand_cap, E_INTERNAL, "peak candidate buffer overflow");
    std::vector<int64_t> idx(n);
    std::vector<float> val(n);
    if (n) {
        TTM_CUDA_TRY(cudaMemcpyAsync(idx.data(), cidx, n * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        TTM_CUDA_TRY(cudaMemcpyAsync(val.data(), cval, n * sizeof(float), cudaMemcpyDeviceToHost, st));
        TTM_CUDA_TRY(cudaStreamSynchronize(st));
    }
    std::vector<int64_t> order(n);
    for (int64_t i = 0; i < (int64_t)n; i++) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t c) {
        if (val[a] != val[c]) return val[a] > val[c];
        return idx[a] < idx[c];
    });
    const double md2 = min_dist * min_dist;
    const int64_t X = p.X, Y = p.Y;
    int got = 0;
    std::vector<double> acc;  // accepted (z, y, x)
    for (int64_t o : order) {
        if (got >= Pk) break;
        int64_t i = idx[o];
        double x = (double)(i % X), y = (double)((i / X) % Y), z = (double)(i / (X * Y));
        bool ok = true;
        for (int a = 0; a < got && ok; a++) {
            double dz = z - acc[3 * a], dy = y - acc[3 * a + 1], dx = x - acc[3 * a + 2];
            if (dz * dz + dy * dy + dx * dx < md2) ok = false;
        }
        if (!ok) continue;
        acc.push_back(z); acc.push_back(y); acc.push_back(x);
        h_idx[got] = i;
        h_val[got] = val[o];
        got++;
    }
    return got;
}

}  // namespace ttm

using namespace ttm;

extern "C" ttm_status ttm_find_peaks(ttm_plan* plan, const float* d_map, int P, double min_dist, int64_t* h_idx,
                                     float* h_val, int* h_count, void* stream)
{
    if (!plan) return TTM_E_INVALID_ARG;
    try {
        TTM_REQUIRE(d_map && h_idx && h_val && h_count && P >= 0 && min_dist >= 0, E_INVALID_ARG, "bad argument");
        TTM_CUDA_TRY(cudaSetDevice(plan->ctx->device));
        *h_count = find_peaks_run(plan, d_map, P, min_dist, h_idx, h_val, (cudaStream_t)stream);
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(plan->ctx, e);
    }
}

// ----------------------------------------------------------------------
// Allocation-free Find Peaks. Same result as ttm_find_peaks, for callers
// that cannot allocate device memory at the point where they need peaks:
// a process whose free device memory is already reserved by another
// allocator (a framework's caching pool that holds the HBM it once used),
// or a streaming loop in which cudaMalloc / cudaFree would synchronise the
// device and stall the work queued on other streams. It also needs no
// plan: ttm_find_peaks takes its candidate buffer from a plan, and
// creating a plan allocates the whole correlate workspace.
//
// The scratch lives in one file-scope device array of fixed size: at most
// kStaticCand local maxima (26-neighbour, inside the box) and at most
// kStaticPeaks accepted peaks. Larger requests are rejected with
// TTM_E_SHAPE. The array is shared by every call on a device, so calls that
// overlap (other streams, other host threads) race on it and must be
// serialised by the caller.
//
// Device work: the compaction kernel above writes the candidates, then one
// CTA repeats "take the best remaining candidate (value desc, index asc),
// remove those closer than min_dist" P times. Taking the best remaining
// candidate that no accepted peak suppresses is exactly the greedy pass over
// the sorted candidate list, so the accepted list equals ttm_find_peaks'.
namespace ttm {

constexpr int64_t kStaticCand = int64_t(1) << 18;  // 262144 candidates
constexpr int kStaticPeaks = 16384;
constexpr size_t kOffCandIdx = 0;                                        // int64 [kStaticCand]
constexpr size_t kOffCandVal = kOffCandIdx + sizeof(int64_t) * kStaticCand;  // float [kStaticCand]
constexpr size_t kOffOutIdx = kOffCandVal + sizeof(float) * kStaticCand;     // int64 [kStaticPeaks]
constexpr size_t kOffOutVal = kOffOutIdx + sizeof(int64_t) * kStaticPeaks;   // float [kStaticPeaks]
constexpr size_t kOffCount = kOffOutVal + sizeof(float) * kStaticPeaks;      // u64 candidate counter
constexpr size_t kOffOutCount = kOffCount + 256;                             // int accepted count
constexpr size_t kStaticScratchBytes = kOffOutCount + 256;                   // 3,342,848 bytes
static_assert(kOffCandVal % 256 == 0 && kOffOutIdx % 256 == 0 && kOffOutVal % 256 == 0 && kOffCount % 256 == 0,
              "scratch parts must stay 256-byte aligned");

static __device__ __align__(256) unsigned char g_peak_scratch[kStaticScratchBytes];

// Device address of g_peak_scratch in the current device's copy of the
// module. Called once per context, at ttm_ctx_create, with the context's
// device current: looking the symbol up loads the module on that device
// (under lazy loading), which commits the array's device memory there and
// then, not inside a later Find Peaks call.
void* peak_scratch_address()
{
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_peak_scratch);
    if (e != cudaSuccess || !p)
        throw Error{E_CUDA, std::string("cudaGetSymbolAddress(peak scratch): ") + cudaGetErrorString(e)};
    return p;
}

// Candidates are kept as packed coordinates z << 42 | y << 21 | x (each
// below 2^21), which order like the linear index (z, y, x lexicographic),
// so the tie rule "lower index first" is unchanged and the distance test
// needs shifts, not 64-bit divisions.
__device__ __forceinline__ int64_t pack_zyx(int64_t i, int64_t X, int64_t Y)
{
    const int64_t x = i % X, r = i / X;
    return ((r / Y) << 42) | ((r % Y) << 21) | x;
}
__device__ __forceinline__ int64_t unpack_index(int64_t c, int64_t X, int64_t Y)
{
    return ((c >> 42) * Y + ((c >> 21) & 0x1FFFFF)) * X + (c & 0x1FFFFF);
}

struct Best {
    float v;
    int64_t i, pos;  // pos < 0: none
};

__device__ __forceinline__ bool better(const Best& a, const Best& b)
{
    if (a.pos < 0) return false;
    if (b.pos < 0) return true;
    if (a.v != b.v) return a.v > b.v;
    return a.i < b.i;
}

__device__ __forceinline__ Best shfl_best(const Best& b, int off)
{
    Best o;
    o.v = __shfl_down_sync(0xffffffffu, b.v, off);
    o.i = __shfl_down_sync(0xffffffffu, b.i, off);
    o.pos = __shfl_down_sync(0xffffffffu, b.pos, off);
    return o;
}

// Greedy selection over the compacted candidates (one CTA). The candidate
// indices are first rewritten as packed coordinates; removed candidates
// get -1. Every kCompactEvery accepted peaks the live candidates are
// compacted in place (stable, one block-wide scan per 1024 entries), so
// later passes only touch survivors. Cost: at most P passes over the live
// candidates, each a few integer operations per candidate; at the caps
// (262 144 candidates, P = 16 384) a pass over all of them is ~0.2 ms on one
// SM, and compaction shrinks the live set as peaks suppress their
// neighbourhoods. *out_count = accepted peaks, or -1 when the candidates
// overflowed the scratch.
constexpr int kCompactEvery = 8;

__global__ void __launch_bounds__(1024) k_select_greedy(const unsigned long long* __restrict__ count, int64_t cap,
                                                        int P, double md2, int64_t X, int64_t Y,
                                                        int64_t* __restrict__ cidx, float* __restrict__ cval,
                                                        int64_t* __restrict__ oidx, float* __restrict__ oval,
                                                        int* __restrict__ out_count)
{
    __shared__ Best warp_best[32];
    __shared__ Best chosen;
    __shared__ int warp_live[32];
    const unsigned long long nn = *count;
    if (nn > (unsigned long long)cap) {
        if (threadIdx.x == 0) *out_count = -1;
        return;
    }
    int64_t n = (int64_t)nn;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) cidx[k] = pack_zyx(cidx[k], X, Y);
    __syncthreads();
    bool have = false;
    int64_t az = 0, ay = 0, ax = 0;
    int got = 0;
    for (int it = 0; it < P; it++) {
        if (it > 0 && it % kCompactEvery == 0) {
            // stable in-place compaction of the live candidates
            int64_t base = 0;
            for (int64_t k0 = 0; k0 < n; k0 += blockDim.x) {
                const int64_t k = k0 + threadIdx.x;
                const int64_t c = k < n ? cidx[k] : -1;
                const float v = k < n ? cval[k] : 0.f;
                const bool live = c >= 0;
                const unsigned ball = __ballot_sync(0xffffffffu, live);
                if (lane == 0) warp_live[warp] = __popc(ball);
                __syncthreads();
                int before = 0, total = 0;
                for (int wi = 0; wi < nwarps; wi++) {
                    if (wi < warp) before += warp_live[wi];
                    total += warp_live[wi];
                }
                before += __popc(ball & ((1u << lane) - 1u));
                __syncthreads();  // every read of this chunk precedes its writes
                if (live) {
                    cidx[base + before] = c;
                    cval[base + before] = v;
                }
                base += total;
                __syncthreads();
            }
            n = base;
        }
        Best b{0.f, 0, -1};
        for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
            const int64_t c = cidx[k];
            if (c < 0) continue;
            if (have) {
                const double dz = (double)((c >> 42) - az), dy = (double)(((c >> 21) & 0x1FFFFF) - ay),
                             dx = (double)((c & 0x1FFFFF) - ax);
                if (dz * dz + dy * dy + dx * dx < md2) {
                    cidx[k] = -1;
                    continue;
                }
            }
            const Best cb{cval[k], c, k};
            if (better(cb, b)) b = cb;
        }
        for (int off = 16; off > 0; off >>= 1) {
            const Best o = shfl_best(b, off);
            if (better(o, b)) b = o;
        }
        if (lane == 0) warp_best[warp] = b;
        __syncthreads();
        if (warp == 0) {
            b = lane < nwarps ? warp_best[lane] : Best{0.f, 0, -1};
            for (int off = 16; off > 0; off >>= 1) {
                const Best o = shfl_best(b, off);
                if (better(o, b)) b = o;
            }
            if (lane == 0) {
                chosen = b;
                if (b.pos >= 0) {
                    oidx[it] = unpack_index(b.i, X, Y);
                    oval[it] = b.v;
                    cidx[b.pos] = -1;
                }
            }
        }
        __syncthreads();
        const Best c = chosen;
        if (c.pos < 0) break;
        got++;
        have = true;
        az = c.i >> 42;
        ay = (c.i >> 21) & 0x1FFFFF;
        ax = c.i & 0x1FFFFF;
        __syncthreads();
    }
    if (threadIdx.x == 0) *out_count = got;
}

}  // namespace ttm

extern "C" ttm_status ttm_find_peaks_noalloc(ttm_ctx* ctx, const float* d_map, int Z, int Y, int X, const int* box,
                                             int P, double min_dist, int64_t* h_idx, float* h_val, int* h_count,
                                             void* stream)
{
    if (!ctx) return TTM_E_INVALID_ARG;
    try {
        TTM_REQUIRE(d_map && box && h_idx && h_val && h_count && Z > 0 && Y > 0 && X > 0 && P >= 0 && min_dist >= 0,
                    E_INVALID_ARG, "bad argument");
        TTM_REQUIRE(box[0] >= 0 && box[0] <= box[1] && box[1] <= Z && box[2] >= 0 && box[2] <= box[3] &&
                        box[3] <= Y && box[4] >= 0 && box[4] <= box[5] && box[5] <= X,
                    E_INVALID_ARG, "box must satisfy 0 <= lo <= hi <= extent on every axis");
        TTM_REQUIRE(P <= kStaticPeaks, E_SHAPE, "P exceeds the static peak capacity of 16384");
        TTM_REQUIRE(Z < (1 << 21) && Y < (1 << 21) && X < (1 << 21), E_SHAPE, "extents must be below 2^21");
        *h_count = 0;
        if (P == 0) return TTM_OK;
        TTM_CUDA_TRY(cudaSetDevice(ctx->device));
        TTM_REQUIRE(ctx->peak_scratch, E_INTERNAL, "context has no peak scratch address");
        unsigned char* s = static_cast<unsigned char*>(ctx->peak_scratch);
        cudaStream_t st = (cudaStream_t)stream;
        int64_t* cidx = reinterpret_cast<int64_t*>(s + kOffCandIdx);
        float* cval = reinterpret_cast<float*>(s + kOffCandVal);
        int64_t* oidx = reinterpret_cast<int64_t*>(s + kOffOutIdx);
        float* oval = reinterpret_cast<float*>(s + kOffOutVal);
        unsigned long long* cnt = reinterpret_cast<unsigned long long*>(s + kOffCount);
        int* ocnt = reinterpret_cast<int*>(s + kOffOutCount);
        // the candidate counter must start at zero on every call
        TTM_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
        k_localmax<<<32 * ctx->num_sms, 256, 0, st>>>(d_map, Z, Y, X, box[0], box[1], box[2], box[3], box[4], box[5],
                                               kStaticCand, cidx, cval, cnt);
        TTM_LAUNCH_CHECK();
        k_select_greedy<<<1, 1024, 0, st>>>(cnt, kStaticCand, P, min_dist * min_dist, X, Y, cidx, cval, oidx, oval,
                                            ocnt);
        TTM_LAUNCH_CHECK();
        int got = 0;
        TTM_CUDA_TRY(cudaMemcpyAsync(&got, ocnt, sizeof(int), cudaMemcpyDeviceToHost, st));
        TTM_CUDA_TRY(cudaStreamSynchronize(st));
        TTM_REQUIRE(got >= 0, E_SHAPE, "more than 262144 local maxima in the box: beyond the static candidate capacity");
        if (got > 0) {
            TTM_CUDA_TRY(cudaMemcpyAsync(h_idx, oidx, got * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            TTM_CUDA_TRY(cudaMemcpyAsync(h_val, oval, got * sizeof(float), cudaMemcpyDeviceToHost, st));
            TTM_CUDA_TRY(cudaStreamSynchronize(st));
        }
        *h_count = got;
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(ctx, e);
    }
}
