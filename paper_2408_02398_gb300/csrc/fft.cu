// fft.cu -- host side of the FFT passes: radix schedules, tile shapes and
// twiddle tables.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "fft.cuh"

namespace ttm {

bool factor_length(int L, LenPlan& pl)
{
    pl.L = L;
    pl.nst = 0;
    pl.tw = nullptr;
    if (L < 1) return false;
    int rest = L;
    // largest radices first; a trailing power of two below 8 becomes one
    // radix-4 or radix-2 stage
    while (rest % 8 == 0 && pl.nst < kMaxStages) { pl.rad[pl.nst++] = 8; rest /= 8; }
    if (rest % 4 == 0) { pl.rad[pl.nst++] = 4; rest /= 4; }
    if (rest % 2 == 0) { pl.rad[pl.nst++] = 2; rest /= 2; }
    const int odd[3] = {7, 5, 3};
    for (int r : odd)
        while (rest % r == 0 && pl.nst < kMaxStages) { pl.rad[pl.nst++] = r; rest /= r; }
    if (L == 1) { pl.rad[pl.nst++] = 2; return false; }
    return rest == 1;
}

TileShape choose_tile(int L, size_t elem_bytes, int min_w, int max_w)
{
    TileShape t;
    // odd line stride (in elements) keeps the W-strided tile loads free of
    // shared-memory bank conflicts for 8- and 16-byte elements
    t.ld = (L % 2 == 0) ? L + 1 : L;
    const size_t budget = 112 * 1024;  // two CTAs per SM
    int W = max_w;
    while (W > min_w && (2 * (size_t)W * t.ld + L) * elem_bytes > budget) W /= 2;
    t.W = W;
    t.smem = (2 * (size_t)W * t.ld + L) * elem_bytes;
    return t;
}

TileShape plan_tile(const LenPlan& pl, size_t elem_bytes, int min_w, int max_w)
{
    if (pl.tile_w >= min_w && pl.tile_w <= max_w) {
        TileShape t;
        t.ld = (pl.L % 2 == 0) ? pl.L + 1 : pl.L;
        t.W = pl.tile_w;
        t.smem = (2 * (size_t)t.W * t.ld + pl.L) * elem_bytes;
        if (t.smem <= 200 * 1024) return t;
    }
    return choose_tile(pl.L, elem_bytes, min_w, max_w);
}

TwiddleCache::~TwiddleCache()
{
    for (int i = 0; i < n_; i++) cudaFree(entries_[i].ptr);
    std::free(entries_);
}

const void* TwiddleCache::get(int L, int kind)
{
    for (int i = 0; i < n_; i++)
        if (entries_[i].L == L && entries_[i].kind == kind) return entries_[i].ptr;
    // exp(-2 pi i m / L) from the exact fraction m / L, in double precision
    std::vector<double> re(L), im(L);
    for (int m = 0; m < L; m++) {
        double a = 2.0 * M_PI * (double)m / (double)L;
        re[m] = std::cos(a);
        im[m] = -std::sin(a);
    }
    void* d = nullptr;
    const size_t esz = kind == TW_F32 ? sizeof(float2) : sizeof(double2);
    const size_t bytes = (size_t)L * esz;
    TTM_CUDA_TRY(cudaMalloc(&d, bytes));
    if (kind == TW_F64) {
        std::vector<double2> h(L);
        for (int m = 0; m < L; m++) h[m] = make_double2(re[m], im[m]);
        TTM_CUDA_TRY(cudaMemcpy(d, h.data(), bytes, cudaMemcpyHostToDevice));
    } else if (kind == TW_DF64) {
        // (re.hi, re.lo, im.hi, im.lo)
        std::vector<float4> h(L);
        for (int m = 0; m < L; m++) {
            float rh = (float)re[m], ih = (float)im[m];
            h[m] = make_float4(rh, (float)(re[m] - (double)rh), ih, (float)(im[m] - (double)ih));
        }
        TTM_CUDA_TRY(cudaMemcpy(d, h.data(), bytes, cudaMemcpyHostToDevice));
    } else {
        std::vector<float2> h(L);
        for (int m = 0; m < L; m++) h[m] = make_float2((float)re[m], (float)im[m]);
        TTM_CUDA_TRY(cudaMemcpy(d, h.data(), bytes, cudaMemcpyHostToDevice));
    }
    if (n_ == cap_) {
        cap_ = cap_ ? 2 * cap_ : 8;
        entries_ = (Entry*)std::realloc(entries_, sizeof(Entry) * cap_);
    }
    entries_[n_++] = Entry{L, kind, d};
    return d;
}

LenPlan make_len_plan(TwiddleCache& tc, int L, int kind)
{
    LenPlan pl;
    TTM_REQUIRE(factor_length(L, pl), E_SHAPE,
                "transform length " + std::to_string(L) + " is not a product of 2, 3, 5 and 7");
    pl.tw = tc.get(L, kind);
    return pl;
}

}  // namespace ttm
