// ttm_blocks.cu -- block processing with halos and Merge Peaks (Sec. 3.4).
// A tomogram in host memory is processed in z-slabs: each slab's output
// planes are a part of the valid z range, and its input carries the
// template's reach on both sides (so every template window of its voxels
// lies inside it), one more plane each side for the 3-tap filter of Eq. 3,
// and its map is evaluated one plane beyond its output planes for the
// 26-neighbour test. Local maxima are taken per slab in its output planes;
// Merge Peaks orders all of them by (value desc, index asc) and accepts
// greedily at the exclusion distance, exactly as Find Peaks does on the
// whole tomogram.
#include <algorithm>
#include <map>
#include <vector>

#include "ttm_internal.h"

namespace ttm {

// candidates at z in [cz0, cz1) (and the y, x box), neighbours tested
// within [nz0, nz1) (and the same y, x box) of a map on a Z x Y x X grid;
// indices written on the tomogram's grid: ((z + zoff) Yt + y) Xt + x
__global__ void k_localmax_slab(const float* __restrict__ s, int Y, int X, int cz0, int cz1, int nz0, int nz1,
                                int y0, int y1, int x0, int x1, int64_t zoff, int Yt, int Xt, int64_t cap,
                                int64_t* __restrict__ idx, float* __restrict__ val,
                                unsigned long long* __restrict__ count)
{
    const int bx = x1 - x0, by = y1 - y0, bz = cz1 - cz0;
    const int64_t n = (int64_t)bx * by * bz;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int x = x0 + (int)(t % bx);
        const int64_t r = t / bx;
        const int y = y0 + (int)(r % by), z = cz0 + (int)(r / by);
        const int64_t i = ((int64_t)z * Y + y) * X + x;
        const float v = s[i];
        if (!(v == v)) continue;
        bool is_max = true;
        for (int dz = -1; dz <= 1 && is_max; dz++)
            for (int dy = -1; dy <= 1 && is_max; dy++)
                for (int dx = -1; dx <= 1 && is_max; dx++) {
                    if (!dz && !dy && !dx) continue;
                    const int zz = z + dz, yy = y + dy, xx = x + dx;
                    if (zz < nz0 || zz >= nz1 || yy < y0 || yy >= y1 || xx < x0 || xx >= x1) continue;
                    const int64_t j = ((int64_t)zz * Y + yy) * X + xx;
                    const float o = s[j];
                    // ties go to the lower linear index; the slab's order of
                    // indices is the tomogram's (same y, x strides per plane)
                    if (o > v || (o == v && j < i)) is_max = false;
                }
        if (!is_max) continue;
        const unsigned long long pos = atomicAdd(count, 1ull);
        if ((int64_t)pos < cap) {
            idx[pos] = (((int64_t)z + zoff) * Yt + y) * Xt + x;
            val[pos] = v;
        }
    }
}

}  // namespace ttm

// A block-processing session: the slab table, one plan per distinct slab
// depth (template spectra on each slab's autotuned working grid), the slab
// buffers and a copy stream, kept from one ttm_blocked_run to the next.
struct ttm_blocked {
    ttm_ctx* ctx = nullptr;
    int Z = 0, Y = 0, X = 0, tz = 0, ty = 0, tx = 0, K = 0, dprime = 3;
    int ns = 0;
    std::vector<int> sl;
    std::map<int, ttm_plan*> plans;
    ttm::DevBuf d_tomo[2], d_C, d_map, d_aux, d_orient, cand, cnt;
    int64_t cap = 0;
    cudaStream_t copy_st = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
    ~ttm_blocked()
    {
        for (auto& kv : plans) ttm_plan_destroy(kv.second);
        for (int b = 0; b < 2; b++) {
            if (copied[b]) cudaEventDestroy(copied[b]);
            if (consumed[b]) cudaEventDestroy(consumed[b]);
        }
        if (copy_st) cudaStreamDestroy(copy_st);
    }
};

using namespace ttm;

extern "C" int ttm_slab_ranges(int Z, int tz, int slab_z, int* out, int cap)
{
    if (Z <= 0 || tz <= 0 || tz > Z || slab_z <= 0) return -1;
    const int cz = tz / 2;
    const int vz0 = cz, vz1 = Z - (tz - cz) + 1;  // valid planes [vz0, vz1)
    int n = 0;
    for (int o0 = vz0; o0 < vz1; o0 += slab_z, n++) {
        if (!out || n >= cap) continue;
        const int o1 = std::min(o0 + slab_z, vz1);
        const int m0 = std::max(vz0, o0 - 1), m1 = std::min(vz1, o1 + 1);
        const int i0 = std::max(0, m0 - cz - 1), i1 = std::min(Z, m1 + (tz - 1 - cz) + 1);
        int* r = out + 6 * n;
        r[0] = o0; r[1] = o1; r[2] = m0; r[3] = m1; r[4] = i0; r[5] = i1;
    }
    return n;
}

extern "C" int ttm_merge_peaks(int64_t n, const int64_t* idx, const float* val, int Z, int Y, int X, int P,
                               double min_dist, int64_t* out_idx, float* out_val)
{
    if (n < 0 || P < 0 || min_dist < 0 || Z <= 0 || Y <= 0 || X <= 0 || (n > 0 && (!idx || !val)) ||
        (P > 0 && (!out_idx || !out_val)))
        return -1;
    std::vector<int64_t> order(n);
    for (int64_t i = 0; i < n; i++) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t c) {
        if (val[a] != val[c]) return val[a] > val[c];
        return idx[a] < idx[c];
    });
    const double md2 = min_dist * min_dist;
    std::vector<double> acc;
    int got = 0;
    for (int64_t o : order) {
        if (got >= P) break;
        const int64_t i = idx[o];
        const double x = (double)(i % X), y = (double)((i / X) % Y), z = (double)(i / ((int64_t)X * Y));
        bool ok = true;
        for (int a = 0; a < got && ok; a++) {
            const double dz = z - acc[3 * a], dy = y - acc[3 * a + 1], dx = x - acc[3 * a + 2];
            if (dz * dz + dy * dy + dx * dx < md2) ok = false;
        }
        if (!ok) continue;
        acc.push_back(z); acc.push_back(y); acc.push_back(x);
        out_idx[got] = i;
        out_val[got] = val[o];
        got++;
    }
    return got;
}

extern "C" ttm_status ttm_blocked_create(ttm_ctx* ctx, const double* d_field, int tz, int ty, int tx,
                                         const ttm_field_params* params, int Z, int Y, int X, int slab_z,
                                         ttm_blocked** out)
{
    if (!ctx) return TTM_E_INVALID_ARG;
    ttm_blocked* B = nullptr;
    try {
        TTM_REQUIRE(d_field && params && out, E_INVALID_ARG, "null pointer argument");
        TTM_REQUIRE(slab_z > 0, E_INVALID_ARG, "slab_z must be positive");
        TTM_REQUIRE(Z >= tz && Y >= ty && X >= tx, E_SHAPE, "tomogram smaller than the template");
        TTM_CUDA_TRY(cudaSetDevice(ctx->device));
        B = new ttm_blocked();
        B->ctx = ctx;
        B->Z = Z; B->Y = Y; B->X = X; B->tz = tz; B->ty = ty; B->tx = tx;
        B->K = ttm_num_components(params->order_n, params->dprime);
        B->dprime = params->dprime;
        B->ns = ttm_slab_ranges(Z, tz, slab_z, nullptr, 0);
        TTM_REQUIRE(B->ns > 0, E_SHAPE, "no valid z plane");
        B->sl.resize(6 * (size_t)B->ns);
        ttm_slab_ranges(Z, tz, slab_z, B->sl.data(), B->ns);
        const int cy = ty / 2, cx = tx / 2;
        const int64_t by = Y - (ty - cy) + 1 - cy, bx = X - (tx - cx) + 1 - cx;
        size_t max_in = 0, max_work = 0;
        for (int s = 0; s < B->ns; s++) {
            const int* r = &B->sl[6 * (size_t)s];
            const int Zs = r[5] - r[4];
            max_in = std::max(max_in, (size_t)Zs * Y * X);
            // strict 26-neighbour maxima: at most one per 2 x 2 x 2 cell
            B->cap += ((r[1] - r[0]) / 2 + 1) * (by / 2 + 1) * (bx / 2 + 1);
            ttm_plan*& plan = B->plans[Zs];
            if (!plan) {
                int work[3];
                const int t3[3] = {Zs, Y, X};
                autotune_shape(ctx, t3, work);
                const ttm_status rc = ttm_plan_create_padded(ctx, d_field, tz, ty, tx, params, Zs, Y, X, work[0],
                                                             work[1], work[2], TTM_PREC_FP32, &plan);
                if (rc != TTM_OK) throw Error{rc, ttm_last_error(ctx)};
            }
            const Prep& p = plan->prep;
            max_work = std::max(max_work, (size_t)p.Z * p.Y * p.X);
        }
        for (int b = 0; b < 2; b++) {
            B->d_tomo[b].alloc(max_in * sizeof(float));
            TTM_CUDA_TRY(cudaEventCreateWithFlags(&B->copied[b], cudaEventDisableTiming));
            TTM_CUDA_TRY(cudaEventCreateWithFlags(&B->consumed[b], cudaEventDisableTiming));
        }
        TTM_CUDA_TRY(cudaStreamCreateWithFlags(&B->copy_st, cudaStreamNonBlocking));
        B->d_C.alloc(max_work * B->K * sizeof(float));
        B->d_map.alloc(max_work * sizeof(float));
        B->d_aux.alloc(max_work * sizeof(float));
        B->d_orient.alloc(max_work * params->dprime * sizeof(float));
        B->cand.alloc((size_t)B->cap * (sizeof(int64_t) + sizeof(float)));
        B->cnt.alloc(sizeof(unsigned long long));
        *out = B;
        return TTM_OK;
    } catch (const Error& e) {
        delete B;
        return (ttm_status)fail(ctx, e);
    }
}

extern "C" void ttm_blocked_destroy(ttm_blocked* b) { delete b; }

extern "C" ttm_status ttm_blocked_run(ttm_blocked* B, const float* h_tomo, int map_kind, int P, double min_dist,
                                      int64_t* h_idx, float* h_val, int* h_count, void* stream)
{
    if (!B) return TTM_E_INVALID_ARG;
    ttm_ctx* ctx = B->ctx;
    try {
        TTM_REQUIRE(h_tomo && h_count && (P == 0 || (h_idx && h_val)), E_INVALID_ARG, "null pointer argument");
        TTM_REQUIRE(P >= 0 && min_dist >= 0 && (map_kind == 0 || map_kind == 1), E_INVALID_ARG,
                    "bad P, min_dist or map_kind");
        TTM_CUDA_TRY(cudaSetDevice(ctx->device));
        cudaStream_t st = (cudaStream_t)stream;
        const int Y = B->Y, X = B->X;
        const int cy = B->ty / 2, cx = B->tx / 2;
        const int y0 = cy, y1 = Y - (B->ty - cy) + 1, x0 = cx, x1 = X - (B->tx - cx) + 1;
        int64_t* cidx = B->cand.as<int64_t>();
        float* cval = reinterpret_cast<float*>(cidx + B->cap);
        TTM_CUDA_TRY(cudaMemsetAsync(B->cnt.p, 0, sizeof(unsigned long long), st));
        for (int b = 0; b < 2; b++) TTM_CUDA_TRY(cudaEventRecord(B->consumed[b], st));
        for (int s = 0; s < B->ns; s++) {
            const int* r = &B->sl[6 * (size_t)s];
            const int o0 = r[0], o1 = r[1], m0 = r[2], m1 = r[3], i0 = r[4], i1 = r[5];
            const int Zs = i1 - i0;
            const int b = s & 1;
            ttm_plan* plan = B->plans.at(Zs);
            // upload of this slab on the copy stream, once the correlation of
            // the slab that last used the buffer has read it
            TTM_CUDA_TRY(cudaStreamWaitEvent(B->copy_st, B->consumed[b], 0));
            TTM_CUDA_TRY(cudaMemcpyAsync(B->d_tomo[b].p, h_tomo + (size_t)i0 * Y * X,
                                         (size_t)Zs * Y * X * sizeof(float), cudaMemcpyHostToDevice, B->copy_st));
            TTM_CUDA_TRY(cudaEventRecord(B->copied[b], B->copy_st));
            TTM_CUDA_TRY(cudaStreamWaitEvent(st, B->copied[b], 0));
            ttm_status rc = ttm_correlate(plan, B->d_tomo[b].as<float>(), B->d_C.as<float>(), stream);
            if (rc != TTM_OK) throw Error{rc, ttm_last_error(ctx)};
            TTM_CUDA_TRY(cudaEventRecord(B->consumed[b], st));
            float* score = map_kind == 0 ? B->d_map.as<float>() : B->d_aux.as<float>();
            float* frob = map_kind == 1 ? B->d_map.as<float>() : B->d_aux.as<float>();
            rc = ttm_peak_map(plan, B->d_C.as<float>(), TTM_MAX_PLAIN, nullptr, score, B->d_orient.as<float>(), frob,
                              stream);
            if (rc != TTM_OK) throw Error{rc, ttm_last_error(ctx)};
            const Prep& p = plan->prep;
            k_localmax_slab<<<32 * B->ctx->num_sms, 256, 0, st>>>(B->d_map.as<float>(), p.Y, p.X, o0 - i0, o1 - i0, m0 - i0,
                                                          m1 - i0, y0, y1, x0, x1, (int64_t)i0, Y, X, B->cap, cidx,
                                                          cval, B->cnt.as<unsigned long long>());
            TTM_LAUNCH_CHECK();
        }
        unsigned long long n = 0;
        TTM_CUDA_TRY(cudaMemcpyAsync(&n, B->cnt.p, sizeof(n), cudaMemcpyDeviceToHost, st));
        TTM_CUDA_TRY(cudaStreamSynchronize(st));
        TTM_REQUIRE((int64_t)n <= B->cap, E_INTERNAL, "peak candidate buffer overflow");
        std::vector<int64_t> li(n);
        std::vector<float> lv(n);
        if (n) {
            TTM_CUDA_TRY(cudaMemcpyAsync(li.data(), cidx, n * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            TTM_CUDA_TRY(cudaMemcpyAsync(lv.data(), cval, n * sizeof(float), cudaMemcpyDeviceToHost, st));
            TTM_CUDA_TRY(cudaStreamSynchronize(st));
        }
        const int got = ttm_merge_peaks((int64_t)n, li.data(), lv.data(), B->Z, Y, X, P, min_dist, h_idx, h_val);
        TTM_REQUIRE(got >= 0, E_INTERNAL, "merge failed");
        *h_count = got;
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(ctx, e);
    }
}

extern "C" ttm_status ttm_blocked_peaks(ttm_ctx* ctx, const double* d_field, int tz, int ty, int tx,
                                        const ttm_field_params* params, const float* h_tomo, int Z, int Y, int X,
                                        int slab_z, int map_kind, int P, double min_dist, int64_t* h_idx,
                                        float* h_val, int* h_count, void* stream)
{
    if (!ctx) return TTM_E_INVALID_ARG;
    if (!h_tomo || !h_count || (P > 0 && (!h_idx || !h_val)) || P < 0 || min_dist < 0 ||
        (map_kind != 0 && map_kind != 1)) {
        ctx->last_error = "bad argument";
        return TTM_E_INVALID_ARG;
    }
    ttm_blocked* B = nullptr;
    ttm_status rc = ttm_blocked_create(ctx, d_field, tz, ty, tx, params, Z, Y, X, slab_z, &B);
    if (rc != TTM_OK) return rc;
    rc = ttm_blocked_run(B, h_tomo, map_kind, P, min_dist, h_idx, h_val, h_count, stream);
    ttm_blocked_destroy(B);
    return rc;
}
