// ttm_peaks.cu -- Find Peaks (Sec. 3.4): local maxima of a score map inside
// the valid box, then the P highest with a minimum exclusion distance.
// The device marks the 26-neighbour maxima (ties go to the lower linear
// index) and compacts them; the host orders the candidates by (value desc,
// index asc) and accepts greedily.
#include <algorithm>
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
    k_localmax<<<4 * 152 * 8, 256, 0, st>>>(d_map, p.Z, p.Y, p.X, b[0], b[1], b[2], b[3], b[4], b[5], P->cand_cap,
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
