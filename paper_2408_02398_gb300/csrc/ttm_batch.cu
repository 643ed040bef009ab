// ttm_batch.cu -- batched TTM: many tomograms of uneven sizes times several
// templates, captured once into one CUDA graph and replayed.
//
// Each tomogram gets a zero-padded working grid (autotuned or the next
// 7-smooth extents) and one preparation (filter, FP64 / double-float local
// sums, spectrum) shared by all of its templates; each (tomogram, template)
// pair keeps its FP32 partial template spectra. The pairs are spread over
// a few branches (streams during capture, parallel paths of the graph),
// balanced by modelled cost; each branch owns one K-component work buffer
// and one C buffer, reused pair after pair, and runs the correlate passes
// and the plain maximiser over the pair's valid box, writing score and
// orientation on the tomogram grid. Small pairs that leave most of the GPU
// idle therefore run side by side, and the whole batch is one graph launch.
#include <algorithm>
#include <memory>
#include <vector>

#include "ttm_internal.h"

namespace ttm {

struct BatchTomo {
    int index = 0;  // position in the caller's list
    const float* d_tomo = nullptr;
    int t[3] = {0, 0, 0};  // tomogram extents
    int w[3] = {0, 0, 0};  // working grid
    int box[6] = {0, 0, 0, 0, 0, 0};
    Prep prep;
    int branch = 0;
    double cost = 0;
    std::vector<int> items;
};

struct BatchItem {
    int tomo = 0, tmpl = 0;
    float *score = nullptr, *orient = nullptr, *frob = nullptr;
    DevBuf spec;
};

static bool smooth7(int L)
{
    if (L < 2) return false;
    for (int r : {2, 3, 5, 7})
        while (L % r == 0) L /= r;
    return L == 1;
}

static int next_smooth7(int n)
{
    int L = std::max(n, 2);
    while (!smooth7(L)) L++;
    return L;
}

}  // namespace ttm

struct ttm_batch {
    ttm_ctx* ctx = nullptr;
    ttm_field_params fp{};
    int K = 0, tz = 0, ty = 0, tx = 0;
    std::vector<std::unique_ptr<ttm::BatchTomo>> tomos;
    std::vector<std::unique_ptr<ttm::BatchItem>> items;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<std::unique_ptr<ttm::DevBuf>> work, cbuf;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~ttm_batch()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (auto e : events) cudaEventDestroy(e);
        for (auto s : streams) cudaStreamDestroy(s);
    }
};

namespace ttm {

static void batch_capture(ttm_batch* B)
{
    const int S = (int)B->streams.size();
    cudaStream_t s0 = B->streams[0];
    TTM_CUDA_TRY(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
    try {
        TTM_CUDA_TRY(cudaEventRecord(B->events[0], s0));
        for (int b = 1; b < S; b++) TTM_CUDA_TRY(cudaStreamWaitEvent(B->streams[b], B->events[0], 0));
        for (auto& tp : B->tomos) {
            BatchTomo& T = *tp;
            if (T.items.empty()) continue;
            cudaStream_t st = B->streams[T.branch];
            prep_filter(T.prep, T.d_tomo, st);
            prep_localsums(T.prep, st);
            prep_spectrum(T.prep, st);
            float2* work = B->work[T.branch]->as<float2>();
            float* C = B->cbuf[T.branch]->as<float>();
            for (int ii : T.items) {
                BatchItem& I = *B->items[ii];
                const DeviceWait dw = B->ctx->wait();
                passes_fp32(T.prep, B->K, I.spec.as<float2>(), work, C, st, &dw);
                peakmap_box_run(B->ctx, B->fp.order_n, C, T.w[0], T.w[1], T.w[2], T.box, T.t[0], T.t[1], T.t[2],
                                I.score, I.orient, I.frob, st);
            }
        }
        for (int b = 1; b < S; b++) {
            TTM_CUDA_TRY(cudaEventRecord(B->events[b], B->streams[b]));
            TTM_CUDA_TRY(cudaStreamWaitEvent(s0, B->events[b], 0));
        }
    } catch (...) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(s0, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    TTM_CUDA_TRY(cudaStreamEndCapture(s0, &B->graph));
    TTM_CUDA_TRY(cudaGraphInstantiate(&B->exec, B->graph, 0));
}

}  // namespace ttm

using namespace ttm;

extern "C" ttm_status ttm_batch_create(ttm_ctx* ctx, const ttm_field_params* params, int tz, int ty, int tx,
                                       int n_templates, const double* const* d_fields, int n_tomos,
                                       const ttm_batch_tomo* tomos, int n_items, const ttm_batch_item* items,
                                       int n_branches, int flags, ttm_batch** out)
{
    if (!ctx) return TTM_E_INVALID_ARG;
    ttm_batch* B = nullptr;
    try {
        TTM_REQUIRE(params && out && d_fields && tomos && items && n_templates > 0 && n_tomos > 0 && n_items > 0,
                    E_INVALID_ARG, "bad argument");
        TTM_REQUIRE(n_branches >= 1 && n_branches <= 16, E_INVALID_ARG, "n_branches must be in 1..16");
        TTM_REQUIRE(params->dprime == 3 && params->order_n >= 2 && params->order_n <= 6 && params->order_n % 2 == 0,
                    E_UNSUPPORTED, "batched TTM is built for d' = 3 and n = 2, 4, 6");
        TTM_REQUIRE(tz > 0 && ty > 0 && tx > 0, E_SHAPE, "bad template shape");
        for (int j = 0; j < n_templates; j++) TTM_REQUIRE(d_fields[j], E_INVALID_ARG, "null field");
        TTM_CUDA_TRY(cudaSetDevice(ctx->device));
        B = new ttm_batch();
        B->ctx = ctx;
        B->fp = *params;
        B->K = ttm_num_components(params->order_n, 3);
        B->tz = tz; B->ty = ty; B->tx = tx;
        for (int i = 0; i < n_tomos; i++) {
            TTM_REQUIRE(tomos[i].d_tomo, E_INVALID_ARG, "null tomogram");
            auto T = std::make_unique<BatchTomo>();
            T->index = i;
            T->d_tomo = tomos[i].d_tomo;
            T->t[0] = tomos[i].Z; T->t[1] = tomos[i].Y; T->t[2] = tomos[i].X;
            TTM_REQUIRE(T->t[0] >= tz && T->t[1] >= ty && T->t[2] >= tx, E_SHAPE, "tomogram smaller than the template");
            if (flags & TTM_BATCH_AUTOTUNE) autotune_shape(ctx, T->t, T->w);
            else for (int a = 0; a < 3; a++) T->w[a] = next_smooth7(T->t[a]);
            prep_create(ctx, T->prep, T->t[0], T->t[1], T->t[2], T->w[0], T->w[1], T->w[2], tz, ty, tx, *params);
            T->prep.localsum_mode = (flags & TTM_BATCH_LOCALSUM_DF64) ? 1 : 0;
            T->box[0] = tz / 2; T->box[1] = T->t[0] - (tz - tz / 2) + 1;
            T->box[2] = ty / 2; T->box[3] = T->t[1] - (ty - ty / 2) + 1;
            T->box[4] = tx / 2; T->box[5] = T->t[2] - (tx - tx / 2) + 1;
            B->tomos.push_back(std::move(T));
        }
        for (int i = 0; i < n_items; i++) {
            const ttm_batch_item& it = items[i];
            TTM_REQUIRE(it.tomo >= 0 && it.tomo < n_tomos && it.tmpl >= 0 && it.tmpl < n_templates, E_INVALID_ARG,
                        "item index out of range");
            TTM_REQUIRE(it.d_score && it.d_orient, E_INVALID_ARG, "null output map");
            auto I = std::make_unique<BatchItem>();
            I->tomo = it.tomo; I->tmpl = it.tmpl;
            I->score = it.d_score; I->orient = it.d_orient; I->frob = it.d_frob;
            BatchTomo& T = *B->tomos[it.tomo];
            const int64_t ncomp = (int64_t)tz * T.w[1] * T.prep.Xh;
            I->spec.alloc(B->K * ncomp * sizeof(float2));
            spectra_fp32(T.prep, B->K, d_fields[it.tmpl], I->spec.as<float2>(), 0);
            T.items.push_back(i);
            B->items.push_back(std::move(I));
        }
        TTM_CUDA_TRY(cudaStreamSynchronize(0));
        // branches balanced by the modelled cost (working voxels x pairs),
        // largest tomograms first
        const int S = std::min(n_branches, n_tomos);
        std::vector<int> order(n_tomos);
        for (int i = 0; i < n_tomos; i++) {
            order[i] = i;
            BatchTomo& T = *B->tomos[i];
            T.cost = (double)T.w[0] * T.w[1] * T.w[2] * (1.0 + (double)T.items.size());
        }
        std::sort(order.begin(), order.end(), [&](int a, int b) { return B->tomos[a]->cost > B->tomos[b]->cost; });
        std::vector<double> load(S, 0.0);
        std::vector<int64_t> need_work(S, 0), need_c(S, 0);
        for (int i : order) {
            BatchTomo& T = *B->tomos[i];
            const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            T.branch = b;
            load[b] += T.cost;
            const int64_t Vw = (int64_t)T.w[0] * T.w[1] * T.w[2];
            if (!T.items.empty()) {
                need_work[b] = std::max(need_work[b], (int64_t)B->K * T.w[0] * T.w[1] * T.prep.Xh);
                need_c[b] = std::max(need_c[b], (int64_t)B->K * Vw);
            }
        }
        // the capture keeps the order of B->tomos: sort them so that each
        // branch issues its tomograms largest first
        std::stable_sort(B->tomos.begin(), B->tomos.end(),
                         [](const std::unique_ptr<BatchTomo>& a, const std::unique_ptr<BatchTomo>& b) {
                             return a->cost > b->cost;
                         });
        for (int b = 0; b < S; b++) {
            cudaStream_t s;
            TTM_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
            B->streams.push_back(s);
            cudaEvent_t e;
            TTM_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            B->events.push_back(e);
            B->work.push_back(std::make_unique<DevBuf>());
            B->cbuf.push_back(std::make_unique<DevBuf>());
            if (need_work[b]) B->work[b]->alloc(need_work[b] * sizeof(float2));
            if (need_c[b]) B->cbuf[b]->alloc(need_c[b] * sizeof(float));
        }
        batch_capture(B);
        *out = B;
        return TTM_OK;
    } catch (const Error& e) {
        delete B;
        return (ttm_status)fail(ctx, e);
    }
}

extern "C" ttm_status ttm_batch_run(ttm_batch* b, void* stream)
{
    if (!b) return TTM_E_INVALID_ARG;
    try {
        TTM_CUDA_TRY(cudaSetDevice(b->ctx->device));
        TTM_CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
        count_launch();
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(b->ctx, e);
    }
}

extern "C" ttm_status ttm_batch_work_shape(const ttm_batch* b, int tomo, int* zyx)
{
    if (!b || !zyx) return TTM_E_INVALID_ARG;
    for (const auto& T : b->tomos)
        if (T->index == tomo) {
            zyx[0] = T->w[0]; zyx[1] = T->w[1]; zyx[2] = T->w[2];
            return TTM_OK;
        }
    return TTM_E_INVALID_ARG;
}

extern "C" void ttm_batch_destroy(ttm_batch* b) { delete b; }
