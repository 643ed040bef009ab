// ttm_api.cu -- context lifetime, errors and small queries of the C ABI.
#include <algorithm>
#include <atomic>
#include <cstring>

#include "ttm_internal.h"

namespace ttm {

void upload_probe_tables(ttm_ctx* ctx);

static std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static cudaEvent_t take_event(ttm_plan* P)
{
    if (!P->free_ev.empty()) {
        cudaEvent_t e = P->free_ev.back();
        P->free_ev.pop_back();
        return e;
    }
    cudaEvent_t e;
    TTM_CUDA_TRY(cudaEventCreate(&e));
    return e;
}

void stage_begin(ttm_plan* P, cudaStream_t st)
{
    if (!P->timing) return;
    P->open_ev = take_event(P);
    TTM_CUDA_TRY(cudaEventRecord(P->open_ev, st));
}

void stage_end(ttm_plan* P, int stage, cudaStream_t st)
{
    if (!P->timing || !P->open_ev) return;
    cudaEvent_t e = take_event(P);
    TTM_CUDA_TRY(cudaEventRecord(e, st));
    P->marks.push_back({stage, P->open_ev, e});
    P->open_ev = e;  // the end of one stage starts the next
}

int fail(ttm_ctx* ctx, const Error& e)
{
    if (ctx) ctx->last_error = e.msg;
    return e.code;
}

}  // namespace ttm

using namespace ttm;

extern "C" void ttm_default_params(ttm_field_params* p)
{
    if (!p) return;
    p->order_n = 4;
    p->dprime = 3;
    p->mask_radius = 16.0;
    p->mask_soft_width = 0.0;
    p->filter_a = 0.2;
    p->n_rot_base = 2048;
    p->cube_symmetrize = 1;
}

extern "C" int ttm_num_components(int n, int d)
{
    if (n < 0 || d < 1) return 0;
    long num = 1, den = 1;
    for (int i = 1; i <= n; i++) { num *= (d - 1 + i); den *= i; }
    return (int)(num / den);
}

extern "C" const char* ttm_version(void) { return "ttm 0.1 sm_103a"; }

extern "C" ttm_status ttm_ctx_create(int device, ttm_ctx** out)
{
    if (!out) return TTM_E_INVALID_ARG;
    ttm_ctx* c = new ttm_ctx();
    c->device = device;
    try {
        TTM_CUDA_TRY(cudaSetDevice(device));
        TTM_CUDA_TRY(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
        upload_probe_tables(c);
        upload_probe_tables4(c);
        c->peak_scratch = peak_scratch_address();
        c->dev_err.alloc(sizeof(int));
        TTM_CUDA_TRY(cudaMemset(c->dev_err.p, 0, sizeof(int)));
        *out = c;
        return TTM_OK;
    } catch (const Error& e) {
        int code = e.code;
        delete c;
        return (ttm_status)code;
    }
}

extern "C" void ttm_ctx_destroy(ttm_ctx* ctx) { delete ctx; }

extern "C" const char* ttm_last_error(const ttm_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

ttm_plan::~ttm_plan()
{
    for (auto& m : marks) { free_ev.push_back(m.a); free_ev.push_back(m.b); }
    if (open_ev) free_ev.push_back(open_ev);
    std::sort(free_ev.begin(), free_ev.end());
    free_ev.erase(std::unique(free_ev.begin(), free_ev.end()), free_ev.end());
    for (cudaEvent_t e : free_ev) cudaEventDestroy(e);
}

static const char* kStageNames[ST_COUNT] = {"prefilter", "image_spectrum", "local_sums", "zpass_fused",
                                            "ypass", "xpass_c2r_norm", "peak_map"};

extern "C" int ttm_num_stages(void) { return ST_COUNT; }

extern "C" const char* ttm_stage_name(int i) { return (i >= 0 && i < ST_COUNT) ? kStageNames[i] : ""; }

extern "C" uint64_t ttm_kernel_launches(void) { return g_launches.load(); }

extern "C" ttm_status ttm_plan_enable_timing(ttm_plan* plan, int on)
{
    if (!plan) return TTM_E_INVALID_ARG;
    plan->timing = on != 0;
    plan->open_ev = nullptr;
    return TTM_OK;
}

extern "C" ttm_status ttm_plan_stage_times(ttm_plan* plan, double* ms, int n)
{
    if (!plan || !ms || n < 0) return TTM_E_INVALID_ARG;
    try {
        for (int i = 0; i < n; i++) ms[i] = 0.0;
        std::vector<cudaEvent_t> used;
        for (auto& m : plan->marks) {
            TTM_CUDA_TRY(cudaEventSynchronize(m.b));
            float t = 0;
            TTM_CUDA_TRY(cudaEventElapsedTime(&t, m.a, m.b));
            if (m.stage < n) ms[m.stage] += t;
            used.push_back(m.a);
            used.push_back(m.b);
        }
        plan->marks.clear();
        if (plan->open_ev) used.push_back(plan->open_ev);
        plan->open_ev = nullptr;
        std::sort(used.begin(), used.end());
        used.erase(std::unique(used.begin(), used.end()), used.end());
        for (cudaEvent_t e : used) plan->free_ev.push_back(e);
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(plan->ctx, e);
    }
}

extern "C" ttm_status ttm_ctx_set_wait_limit(ttm_ctx* ctx, int64_t polls)
{
    if (!ctx || polls < 0) return TTM_E_INVALID_ARG;
    ctx->wait_limit = (long long)polls;
    return TTM_OK;
}

extern "C" ttm_status ttm_ctx_device_status(ttm_ctx* ctx, void* stream)
{
    if (!ctx) return TTM_E_INVALID_ARG;
    try {
        TTM_CUDA_TRY(cudaSetDevice(ctx->device));
        cudaStream_t st = (cudaStream_t)stream;
        int flag = 0;
        TTM_CUDA_TRY(cudaMemcpyAsync(&flag, ctx->dev_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        TTM_CUDA_TRY(cudaStreamSynchronize(st));
        if (!flag) return TTM_OK;
        TTM_CUDA_TRY(cudaMemsetAsync(ctx->dev_err.p, 0, sizeof(int), st));
        TTM_CUDA_TRY(cudaStreamSynchronize(st));
        throw Error{E_TIMEOUT, "a bounded device wait expired: the outputs of the calls since the last check are "
                               "undefined"};
    } catch (const Error& e) {
        return (ttm_status)fail(ctx, e);
    }
}
