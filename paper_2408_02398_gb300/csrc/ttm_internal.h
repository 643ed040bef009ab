// ttm_internal.h -- context and plan objects behind the C ABI of include/ttm.h.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/ttm.h"
#include "fft.cuh"

namespace ttm {

// Device buffer owned by a context or plan (freed in the destructor).
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void alloc(size_t n);
    void release();
    template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

// Per-tomogram-shape workspace shared by the TTM correlate and the TM
// baseline: filtered tomogram, its spectrum, FP64 local sums and w.
struct Prep {
    int Zt = 0, Yt = 0, Xt = 0;  // tomogram
    int Z = 0, Y = 0, X = 0, Xh = 0;  // working grid (>= tomogram; zero padded)
    int tz = 0, ty = 0, tx = 0;
    double M = 0;              // sum of the mask
    double filter_a = 0.2;
    int64_t nblk_pre = 0;      // blocks of the prefilter reduction
    DevBuf g32;                // float [Z][Y][X] filtered tomogram g
    DevBuf G;                  // float2 [Z][Y][Xh] spectrum of g
    DevBuf zc;                 // double2 [Z][Y][X]: (g, g^2), transformed in place
    DevBuf mhat;               // double [(Z/2+1)][(Y/2+1)][(X/2+1)] mask spectrum / V
    DevBuf w;                  // float [Z][Y][X] local normaliser
    DevBuf partials;           // double [2][nblk_pre]
    DevBuf floor;              // double [1]: variance floor
    DevBuf mask_t;             // double [tz][ty][tx] mask on the template grid
    DevBuf mhat_df;            // float2 (hi, lo) copy of mhat for the double-float sums
    int localsum_mode = 0;     // 0: FP64, 1: double-float (FP32 pairs)
    LenPlan px32, py32, pz32, px64, py64, pz64, pxd, pyd, pzd;
};

void prep_create(ttm_ctx* ctx, Prep& p, int Zt, int Yt, int Xt, int Z, int Y, int X, int tz, int ty, int tx,
                 const ttm_field_params& fp);
// the three parts of the per-tomogram preparation, in this order:
// g = h * f (+ variance floor), G = FFT(g), FP64 local sums -> w
void prep_filter(Prep& p, const float* d_tomo, cudaStream_t st);
void prep_spectrum(Prep& p, cudaStream_t st);
void prep_localsums(Prep& p, cudaStream_t st);

// CUDA-event stage timing of a plan (no-ops while timing is off)
enum Stage { ST_FILTER = 0, ST_SPECTRUM, ST_LOCALSUM, ST_ZCORR, ST_YPASS, ST_XPASS, ST_PEAKMAP, ST_COUNT };
void stage_begin(ttm_plan* P, cudaStream_t st);
void stage_end(ttm_plan* P, int stage, cudaStream_t st);

// bounded device waits: the context's sticky error word and poll limit
struct DeviceWait {
    int* err = nullptr;
    long long limit = 0;
};

// fused z pass of the correlation (spectrum / output storage float2, or
// FP16 / BF16 pairs with the image spectrum scaled by 1 / *gmax); with a
// DeviceWait, the TMA-staged kernel where it applies (register length
// <= 256, row strides a multiple of 16 bytes)
template <typename TS, typename TW>
void launch_zcorr(const float2* G, const TS* spec, int K, int tzn, int cz, int64_t ncols, TW* out,
                  const LenPlan& pz, const float* gmax, float oscale, cudaStream_t st,
                  const DeviceWait* dw = nullptr);
template <typename TS, typename TW>
bool launch_zcorr_tma(const float2* G, const TS* spec, int K, int tzn, int cz, int64_t ncols, TW* out,
                      const LenPlan& pz, const float* gmax, float oscale, const DeviceWait& dw, cudaStream_t st);

// FP32 partial template spectra (K components) on the grid of p, and the
// three K-component passes of the FP32 correlate into C [K][Z][Y][X]
void spectra_fp32(Prep& p, int K, const double* d_field, float2* spec, cudaStream_t st);
void passes_fp32(Prep& p, int K, const float2* spec, float2* work, float* C, cudaStream_t st,
                 const DeviceWait* dw = nullptr);
// plain maximiser over box b of C (grid Z x Yin x Xin), maps written on a
// Zo x Yout x Xout grid at the same coordinates
void peakmap_box_run(ttm_ctx* ctx, int n, const float* C, int Z, int Yin, int Xin, const int* b, int Zo, int Yout,
                     int Xout, float* score, float* orient, float* frob, cudaStream_t st);
void autotune_shape(ttm_ctx* ctx, const int t[3], int out[3]);

// LenPlan of length L and twiddle kind: the autotuned schedule and tile
// width when the context has one for FP32 L, else the default schedule;
// for double-float L the register / shared-memory choice is timed on first
// use and kept in the context
LenPlan ctx_len_plan(ttm_ctx* ctx, int L, int kind);

// host mask on the template grid (Sec. 2 after Eq. 3); returns M
double make_mask(int tz, int ty, int tx, double r, double soft, std::vector<double>& m);

// the rotation quadrature of Eq. 9 (n_base super-Fibonacci quaternions,
// optionally times the 24 cube rotations) and the graded-lex descending
// exponents of (w, x, y, z) with sum n (4 per component)
void rotation_set(int64_t n_base, bool cube, std::vector<double>& q);
// t' of Eq. 4 (filter, mask, zero mean and unit norm under the mask) of a
// raw float template, FP64 on the device, returned in tp
void normalise_template_dev(ttm_ctx* ctx, const float* d_tmpl, int tz, int ty, int tx, const ttm_field_params& fp,
                            DevBuf& tp, cudaStream_t st);
void exponents4(int n, std::vector<int>& e);
// device address of the fixed scratch array of the allocation-free Find
// Peaks on the current device (looked up once per context)
void* peak_scratch_address();
// probe tables of the quaternion maximiser, and the maximiser itself over
// all V voxels (orient: [4][V] unit quaternions)
void upload_probe_tables4(ttm_ctx* ctx);
void peakmap4_run(ttm_ctx* ctx, int n, const float* C, int64_t V, float* score, float* orient, float* frob,
                  cudaStream_t st);

}  // namespace ttm

namespace ttm {
// one autotuned FP32 transform length: the fastest of the register kernel
// and the shared-memory passes over radix schedules and tile widths
struct TuneRec {
    int L = 0;
    int kind = 0; // TW_F32 or TW_DF64 passes
    int reg = 0;  // 1: register kernel
    int W = 0;    // tile width of the shared-memory passes
    int nst = 0;
    int rad[kMaxStages] = {};
    double us_line = 0;  // measured microseconds per line of a strided pass
};
}  // namespace ttm

struct ttm_ctx {
    int device = 0;
    std::vector<ttm::TuneRec> tune;  // autotuner cache
    std::string last_error;
    ttm::TwiddleCache twiddles;
    int num_sms = 0;
    ttm::DevBuf probe_tables;  // maximiser probe directions and monomials
    size_t probe_off[5] = {0, 0, 0, 0, 0};
    ttm::DevBuf probe_half;    // FP16 monomial tables for the tensor-core probe product
    size_t probe_half_off[3] = {0, 0, 0};
    ttm::DevBuf probe4;        // quaternion maximiser: probe quaternions and FP16 monomials
    size_t probe4_off[4] = {0, 0, 0, 0};
    void* peak_scratch = nullptr;  // device address of the allocation-free Find Peaks scratch
    // sticky record of an expired bounded device wait (int, device) and the
    // poll limit of such waits
    ttm::DevBuf dev_err;
    long long wait_limit = 1ll << 22;
    ttm::DeviceWait wait() { return ttm::DeviceWait{dev_err.as<int>(), wait_limit}; }
};

struct ttm_plan {
    ttm_ctx* ctx = nullptr;
    ttm_field_params fp{};
    int K = 0;
    ttm_precision prec = TTM_PREC_FP32;
    ttm::Prep prep;
    ttm::DevBuf spec;        // [K][tz][Y][Xh] partial template spectra (x,y transformed)
    ttm::DevBuf spec_scale;  // float [K]: output factor 1 / (s_alpha q) of the 16-bit spectra
    ttm::DevBuf gmax;        // float [1]: max |G| of the last image spectrum (16-bit spectra)
    float work_qz = 1.f;     // factor applied at the z-pass store (16-bit spectra)
    float work_q = 1.f;      // factor applied at the y-pass store (16-bit spectra)
    ttm::DevBuf work;        // [K][Z][Y][Xh] complex: float2, or FP16 / BF16 pairs
    ttm::DevBuf cand;        // peak candidates
    ttm::DevBuf cand_count;  // unsigned long long [1]
    ttm::DevBuf fb_count;    // unsigned long long [1]: learned-maximiser fallbacks of the last call
    int64_t cand_cap = 0;
    // stage timing
    bool timing = false;
    cudaEvent_t open_ev = nullptr;
    struct Mark { int stage; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> free_ev;
    ~ttm_plan();
};

// the warm-start MLP: FP32 parameters with Adam state, training scratch,
// and the BF16 image used by the tensor-core inference
struct ttm_mlp {
    ttm_ctx* ctx = nullptr;
    int K = 0;
    int64_t np = 0;
    int64_t step = 0;
    ttm::DevBuf params, grad, m, v;
    int64_t cap = 0;  // rows of training scratch
    ttm::DevBuf xb, ub, a1, h1, a2, h2, y, dy, loss, part;
    ttm::DevBuf image;         // kMlpImageBytes, rebuilt when the parameters change
    bool image_dirty = true;
    bool bf16 = false;         // forward / backward products in BF16 (tensor cores)
};

namespace ttm {
// set the context error text and return the code
int fail(ttm_ctx* ctx, const Error& e);
// rebuild the BF16 inference image if the parameters changed (synchronous)
void mlp_refresh_image(ttm_mlp* M);
}
