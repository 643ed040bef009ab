// ttm_autotune.cu -- FFT autotuner: for each FP32 transform length it times
// the register kernel (where one exists) and the shared-memory Stockham
// passes over a set of radix schedules and tile widths, on a strided pass
// of 4096 lines, and keeps the fastest. Working-grid shapes for tomograms of
// any size are then chosen among the 7-smooth lengths a little above each
// extent by the modelled cost of the transform passes, and the records can
// be saved to / loaded from a JSON file.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fft_reg.cuh"
#include "ttm_internal.h"

namespace ttm {

namespace {

constexpr int kTuneLines = 4096;
constexpr double kShapeSlack = 1.34;  // largest working extent / tomogram extent considered
constexpr int kMaxLenCandidates = 10;

bool smooth7(int L)
{
    if (L < 2) return false;
    for (int r : {2, 3, 5, 7})
        while (L % r == 0) L /= r;
    return L == 1;
}

// radix schedules: the power-of-two part as {8, 4, 2} multisets with at
// most one 2 and two 4s, in descending and ascending order, with the odd
// radices before or after it
std::vector<std::vector<int>> schedules(int L)
{
    int a = 0, rest = L;
    while (rest % 2 == 0) { rest /= 2; a++; }
    std::vector<int> odd;
    for (int r : {7, 5, 3})
        while (rest % r == 0) { odd.push_back(r); rest /= r; }
    std::vector<std::vector<int>> p2;
    for (int n2 = 0; n2 <= 1; n2++)
        for (int n4 = 0; n4 <= 2; n4++) {
            const int e = a - n2 - 2 * n4;
            if (e < 0 || e % 3) continue;
            std::vector<int> v(e / 3, 8);
            for (int i = 0; i < n4; i++) v.push_back(4);
            for (int i = 0; i < n2; i++) v.push_back(2);
            p2.push_back(v);
            std::vector<int> asc(v.rbegin(), v.rend());
            if (asc != v) p2.push_back(asc);
        }
    std::vector<std::vector<int>> out;
    for (const auto& v : p2) {
        std::vector<int> s1 = v;
        s1.insert(s1.end(), odd.begin(), odd.end());
        out.push_back(s1);
        if (!odd.empty() && !v.empty()) {
            std::vector<int> s2 = odd;
            s2.insert(s2.end(), v.begin(), v.end());
            out.push_back(s2);
        }
    }
    return out;
}

double time_pass(float2* buf, const LenPlan& pl, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1)
{
    const StridedAxis ax{kTuneLines, 1, 0, kTuneLines};
    auto run = [&]() {
        launch_strided_any<float, -1>(buf, ax, pl, ProIdentity<float>(), StoreTo<float>{buf, 0, kTuneLines}, st);
    };
    for (int i = 0; i < 2; i++) run();
    TTM_CUDA_TRY(cudaEventRecord(e0, st));
    const int reps = 5;
    for (int i = 0; i < reps; i++) run();
    TTM_CUDA_TRY(cudaEventRecord(e1, st));
    TTM_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    TTM_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    return 1000.0 * ms / reps / kTuneLines;
}

const TuneRec* find_rec(const ttm_ctx* ctx, int L, int kind = TW_F32)
{
    for (const auto& r : ctx->tune)
        if (r.L == L && r.kind == kind) return &r;
    return nullptr;
}

// Double-float passes: the register four-step against the shared-memory
// Stockham pass (default schedule and tile), timed on a strided pass over a
// buffer of at least 256 MB, so that it runs from DRAM as the local sums do
// (from L2 the register kernel's low occupancy hides and it wins where it
// loses in place). Register pressure and shared memory per CTA differ a lot
// with the length (32 double-float complex values per thread at 512 and
// 1024), and the faster one was measured to change with it.
int tune_lines_df(int L)
{
    const int64_t want = ((int64_t)1 << 28) / ((int64_t)L * (int64_t)sizeof(dcx));
    return (int)std::max<int64_t>(4096, (want + 1023) / 1024 * 1024);
}

double time_pass_df(dcx* buf, int lines, const LenPlan& pl, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1)
{
    const StridedAxis ax{lines, 1, 0, lines};
    auto run = [&]() {
        launch_strided_any<df64, -1>(buf, ax, pl, ProIdentity<df64>(), StoreTo<df64>{buf, 0, lines}, st);
    };
    for (int i = 0; i < 2; i++) run();
    TTM_CUDA_TRY(cudaEventRecord(e0, st));
    const int reps = 4;
    for (int i = 0; i < reps; i++) run();
    TTM_CUDA_TRY(cudaEventRecord(e1, st));
    TTM_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    TTM_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    return 1000.0 * ms / reps / lines;
}

const TuneRec& tune_length_df(ttm_ctx* ctx, int L)
{
    if (const TuneRec* r = find_rec(ctx, L, TW_DF64)) return *r;
    TuneRec rec;
    rec.L = L;
    rec.kind = TW_DF64;
    LenPlan base = make_len_plan(ctx->twiddles, L, TW_DF64);
    rec.nst = base.nst;
    std::copy(base.rad, base.rad + base.nst, rec.rad);
    int E, P;
    if (line3_length(L)) {
        // the three-level register kernel: twice as fast as the shared-memory
        // pass at 512 and 200, so no timing (which also keeps the choice
        // the same under a profiler, whose per-launch overhead evens out the
        // two timings)
        rec.reg = 1;
    } else if (fs_split(L, E, P)) {
        const int lines = tune_lines_df(L);
        DevBuf buf;
        buf.alloc((size_t)L * lines * sizeof(dcx));
        TTM_CUDA_TRY(cudaMemset(buf.p, 0, buf.bytes));
        cudaStream_t st;
        cudaEvent_t e0, e1;
        TTM_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        TTM_CUDA_TRY(cudaEventCreate(&e0));
        TTM_CUDA_TRY(cudaEventCreate(&e1));
        double t_reg = 1e30, t_smem = 1e30;
        try {
            // two interleaved measurements of each, the faster of each kept
            LenPlan sm = base;
            sm.no_reg = 1;
            for (int r = 0; r < 2; r++) {
                t_reg = std::min(t_reg, time_pass_df(buf.as<dcx>(), lines, base, st, e0, e1));
                t_smem = std::min(t_smem, time_pass_df(buf.as<dcx>(), lines, sm, st, e0, e1));
            }
        } catch (...) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            cudaStreamDestroy(st);
            throw;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaStreamDestroy(st);
        // the register kernel only when clearly faster: in the local sums
        // the shared-memory pass won at 512 (7.35 against 8.14 ms on
        // 512 x 512 x 200) where an isolated pass had the two within noise,
        // and the register kernel at 1024 (48.4 against 50.1 ms on
        // 1024 x 1024 x 256)
        rec.reg = t_reg < 0.95 * t_smem ? 1 : 0;
        rec.us_line = std::min(t_reg, t_smem);
    }
    ctx->tune.push_back(rec);
    return ctx->tune.back();
}

const TuneRec& tune_length(ttm_ctx* ctx, int L)
{
    if (const TuneRec* r = find_rec(ctx, L)) return *r;
    TTM_REQUIRE(smooth7(L), E_SHAPE, "autotuner: length is not 7-smooth");
    DevBuf buf;
    buf.alloc((size_t)L * kTuneLines * sizeof(float2));
    TTM_CUDA_TRY(cudaMemset(buf.p, 0, buf.bytes));
    cudaStream_t st;
    cudaEvent_t e0, e1;
    TTM_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    TTM_CUDA_TRY(cudaEventCreate(&e0));
    TTM_CUDA_TRY(cudaEventCreate(&e1));
    TuneRec best;
    best.L = L;
    best.us_line = 1e30;
    try {
        LenPlan base = make_len_plan(ctx->twiddles, L, TW_F32);
        int E, P;
        if (fs_split(L, E, P)) {
            const double t = time_pass(buf.as<float2>(), base, st, e0, e1);
            if (t < best.us_line) {
                best.us_line = t;
                best.reg = 1;
                best.W = 0;
                best.nst = base.nst;
                std::copy(base.rad, base.rad + base.nst, best.rad);
            }
        }
        for (const auto& sch : schedules(L)) {
            if ((int)sch.size() > kMaxStages) continue;
            LenPlan pl = base;
            pl.no_reg = 1;
            pl.nst = (int)sch.size();
            std::copy(sch.begin(), sch.end(), pl.rad);
            for (int W : {4, 8, 16}) {
                pl.tile_w = W;
                if (plan_tile(pl, sizeof(float2), 4, 16).W != W) continue;
                const double t = time_pass(buf.as<float2>(), pl, st, e0, e1);
                if (t < best.us_line) {
                    best.us_line = t;
                    best.reg = 0;
                    best.W = W;
                    best.nst = pl.nst;
                    std::copy(pl.rad, pl.rad + pl.nst, best.rad);
                }
            }
        }
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaStreamDestroy(st);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    ctx->tune.push_back(best);
    return ctx->tune.back();
}

// smallest 7-smooth lengths in [n, kShapeSlack n]
std::vector<int> length_candidates(int n)
{
    std::vector<int> c;
    const int hi = std::max(n, (int)(kShapeSlack * n));
    for (int L = std::max(n, 2); L <= hi && (int)c.size() < kMaxLenCandidates; L++)
        if (smooth7(L)) c.push_back(L);
    if (c.empty()) {
        int L = std::max(n, 2);
        while (!smooth7(L)) L++;
        c.push_back(L);
    }
    return c;
}

}  // namespace

LenPlan ctx_len_plan(ttm_ctx* ctx, int L, int kind)
{
    LenPlan pl = make_len_plan(ctx->twiddles, L, kind);
    if (kind == TW_DF64) {
        pl.no_reg = tune_length_df(ctx, L).reg ? 0 : 1;
        return pl;
    }
    if (kind != TW_F32) return pl;
    const TuneRec* r = find_rec(ctx, L);
    if (!r) return pl;
    pl.no_reg = r->reg ? 0 : 1;
    pl.tile_w = r->W;
    pl.nst = r->nst;
    std::copy(r->rad, r->rad + r->nst, pl.rad);
    return pl;
}

// working grid for a Zt x Yt x Xt tomogram: minimises the modelled cost of
// the transform passes, V_work * sum over axes of (time per line / L)
void autotune_shape(ttm_ctx* ctx, const int t[3], int out[3])
{
    std::vector<int> cand[3];
    std::vector<double> cost[3];
    for (int a = 0; a < 3; a++) {
        cand[a] = length_candidates(t[a]);
        for (int L : cand[a]) cost[a].push_back(tune_length(ctx, L).us_line / L);
    }
    double best = 1e300;
    for (size_t i = 0; i < cand[0].size(); i++)
        for (size_t j = 0; j < cand[1].size(); j++)
            for (size_t k = 0; k < cand[2].size(); k++) {
                const double V = (double)cand[0][i] * cand[1][j] * cand[2][k];
                const double c = V * (cost[0][i] + cost[1][j] + cost[2][k]);
                if (c < best) {
                    best = c;
                    out[0] = cand[0][i];
                    out[1] = cand[1][j];
                    out[2] = cand[2][k];
                }
            }
}

}  // namespace ttm

using namespace ttm;

extern "C" ttm_status ttm_autotune_shape(ttm_ctx* ctx, int Z, int Y, int X, int* zyx)
{
    if (!ctx || !zyx || Z < 1 || Y < 1 || X < 1) return TTM_E_INVALID_ARG;
    try {
        TTM_CUDA_TRY(cudaSetDevice(ctx->device));
        const int t[3] = {Z, Y, X};
        autotune_shape(ctx, t, zyx);
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(ctx, e);
    }
}

extern "C" int ttm_autotune_entries(const ttm_ctx* ctx) { return ctx ? (int)ctx->tune.size() : 0; }

extern "C" ttm_status ttm_autotune_save(const ttm_ctx* ctx, const char* path)
{
    if (!ctx || !path) return TTM_E_INVALID_ARG;
    FILE* f = std::fopen(path, "w");
    if (!f) return TTM_E_INVALID_ARG;
    std::fprintf(f, "[\n");
    for (size_t i = 0; i < ctx->tune.size(); i++) {
        const TuneRec& r = ctx->tune[i];
        std::fprintf(f, "  {\"L\": %d, \"kind\": %d, \"reg\": %d, \"W\": %d, \"rad\": [", r.L, r.kind, r.reg, r.W);
        for (int s = 0; s < r.nst; s++) std::fprintf(f, "%s%d", s ? ", " : "", r.rad[s]);
        std::fprintf(f, "], \"us_line\": %.6g}%s\n", r.us_line, i + 1 < ctx->tune.size() ? "," : "");
    }
    std::fprintf(f, "]\n");
    return std::fclose(f) == 0 ? TTM_OK : TTM_E_INTERNAL;
}

// reads the records written by ttm_autotune_save (one object per line);
// entries for lengths already tuned are replaced
extern "C" ttm_status ttm_autotune_load(ttm_ctx* ctx, const char* path)
{
    if (!ctx || !path) return TTM_E_INVALID_ARG;
    FILE* f = std::fopen(path, "r");
    if (!f) return TTM_E_INVALID_ARG;
    char line[1024];
    std::vector<TuneRec> recs;
    bool ok = true;
    while (std::fgets(line, sizeof line, f)) {
        const char* p = std::strstr(line, "\"L\"");
        if (!p) continue;
        TuneRec r;
        const char* q = std::strstr(line, "\"rad\": [");
        const char* u = std::strstr(line, "\"us_line\":");
        if (!q || !u || std::sscanf(p, "\"L\": %d, \"kind\": %d, \"reg\": %d, \"W\": %d", &r.L, &r.kind, &r.reg,
                                    &r.W) != 4 ||
            std::sscanf(u, "\"us_line\": %lf", &r.us_line) != 1) {
            ok = false;
            break;
        }
        q += 8;
        int prod = 1;
        while (*q && *q != ']' && r.nst < kMaxStages) {
            int v = 0, adv = 0;
            if (std::sscanf(q, " %d%n", &v, &adv) != 1) break;
            r.rad[r.nst++] = v;
            prod *= v;
            q += adv;
            while (*q == ',' || *q == ' ') q++;
        }
        bool radix_ok = true;
        for (int s = 0; s < r.nst; s++)
            radix_ok &= (r.rad[s] == 2 || r.rad[s] == 3 || r.rad[s] == 4 || r.rad[s] == 5 || r.rad[s] == 7 ||
                         r.rad[s] == 8);
        if (r.L < 2 || prod != r.L || !radix_ok || (r.reg != 0 && r.reg != 1) || r.W < 0 || r.W > 16 ||
            (r.kind != TW_F32 && r.kind != TW_DF64)) {
            ok = false;
            break;
        }
        recs.push_back(r);
    }
    std::fclose(f);
    if (!ok) return TTM_E_INVALID_ARG;
    for (const auto& r : recs) {
        bool replaced = false;
        for (auto& e : ctx->tune)
            if (e.L == r.L && e.kind == r.kind) { e = r; replaced = true; }
        if (!replaced) ctx->tune.push_back(r);
    }
    return TTM_OK;
}
