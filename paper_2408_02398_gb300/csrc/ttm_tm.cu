// ttm_tm.cu -- classical template matching baseline (Eqs. 1, 6, 7): for
// every rotation R_j, c(x, R_j) = w(x) (g * t'_{R_j})(x), keeping the
// running maximum and the first rotation index that attains it.
//
// Per rotation: the rotated template t'(R^T p) (trilinear, FP64 sample
// stored FP32) is transformed along x and y on its own z rows, then the
// same fused z pass as the tensorial correlation (one component), a y pass
// and a complex-to-real x pass whose epilogue updates the maximum.
#include <cmath>
#include <vector>

#include "fft_reg.cuh"
#include "ttm_internal.h"

namespace ttm {


void normalise_template_dev(ttm_ctx* ctx, const float* d_tmpl, int tz, int ty, int tx,
                            const ttm_field_params& fp, DevBuf& tp, cudaStream_t st);

struct Rot9 { double r[9]; };

__global__ void k_rotate_template(const double* __restrict__ tp, int tz, int ty, int tx, Rot9 R, double scale,
                                  float* __restrict__ out)
{
    const int n = tz * ty * tx;
    const int cz = tz / 2, cy = ty / 2, cx = tx / 2;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int x = v % tx, y = (v / tx) % ty, z = v / (tx * ty);
        double px = x - cx, py = y - cy, pz = z - cz;
        double sx = R.r[0] * px + R.r[3] * py + R.r[6] * pz + cx;
        double sy = R.r[1] * px + R.r[4] * py + R.r[7] * pz + cy;
        double sz = R.r[2] * px + R.r[5] * py + R.r[8] * pz + cz;
        double x0 = floor(sx), y0 = floor(sy), z0 = floor(sz);
        double ax = sx - x0, ay = sy - y0, az = sz - z0;
        double acc = 0;
        for (int dz = 0; dz <= 1; dz++)
            for (int dy = 0; dy <= 1; dy++)
                for (int dx = 0; dx <= 1; dx++) {
                    int xx = (int)x0 + dx, yy = (int)y0 + dy, zz = (int)z0 + dz;
                    if (xx < 0 || xx >= tx || yy < 0 || yy >= ty || zz < 0 || zz >= tz) continue;
                    acc += (dx ? ax : 1 - ax) * (dy ? ay : 1 - ay) * (dz ? az : 1 - az) * tp[(zz * ty + yy) * tx + xx];
                }
        out[v] = (float)(acc * scale);
    }
}

struct SrcTemplateRows {
    const float* t;
    int Y, X, ty, tx;
    __device__ float operator()(int64_t row, int x) const
    {
        int j = (int)(row / Y), y = (int)(row - (int64_t)j * Y);
        int iy = wrap_to_template(y, Y, ty), ix = wrap_to_template(x, X, tx);
        if (iy < 0 || ix < 0) return 0.f;
        return t[((int64_t)j * ty + iy) * tx + ix];
    }
};

struct SinkTMMax {
    const float* w;
    float* best;
    int32_t* best_idx;
    int X;
    int32_t j;
    __device__ void operator()(int, int64_t row, int x, float v) const
    {
        int64_t i = row * X + x;
        float c = __ldg(w + i) * v;
        if (c > best[i]) { best[i] = c; best_idx[i] = j; }
    }
};

__global__ void k_tm_init(float* best, int32_t* idx, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        best[i] = -INFINITY;
        idx[i] = -1;
    }
}

}  // namespace ttm

using namespace ttm;

extern "C" ttm_status tm_correlate(ttm_ctx* ctx, const float* d_tomo, int Z, int Y, int X, const float* d_tmpl,
                                   int tz, int ty, int tx, const ttm_field_params* params, const double* h_quats,
                                   int64_t n_rot, float* d_best, int32_t* d_best_idx, void* stream)
{
    if (!ctx) return TTM_E_INVALID_ARG;
    try {
        TTM_REQUIRE(d_tomo && d_tmpl && params && h_quats && d_best && d_best_idx, E_INVALID_ARG,
                    "null pointer argument");
        TTM_REQUIRE(n_rot > 0 && n_rot < (1ll << 31), E_INVALID_ARG, "n_rot out of range");
        TTM_REQUIRE(params->mask_radius > 0 && params->filter_a >= 0 && params->filter_a < 0.25, E_INVALID_ARG,
                    "bad mask radius or filter parameter");
        TTM_CUDA_TRY(cudaSetDevice(ctx->device));
        cudaStream_t st = (cudaStream_t)stream;
        Prep p;
        prep_create(ctx, p, Z, Y, X, Z, Y, X, tz, ty, tx, *params);
        DevBuf tp;
        normalise_template_dev(ctx, d_tmpl, tz, ty, tx, *params, tp, st);
        const int Xh = p.Xh;
        const int64_t ncols = (int64_t)Y * Xh, V = (int64_t)Z * Y * X;
        DevBuf rot, part, work;
        rot.alloc((size_t)tz * ty * tx * sizeof(float));
        part.alloc((size_t)tz * ncols * sizeof(float2));
        work.alloc((size_t)Z * ncols * sizeof(float2));
        prep_filter(p, d_tomo, st);
        prep_spectrum(p, st);
        prep_localsums(p, st);
        k_tm_init<<<1024, 256, 0, st>>>(d_best, d_best_idx, V);
        TTM_LAUNCH_CHECK();
        float2* pt = part.as<float2>();
        float2* wk = work.as<float2>();
        for (int64_t j = 0; j < n_rot; j++) {
            const double* q = h_quats + 4 * j;
            double nq = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
            TTM_REQUIRE(nq > 0, E_INVALID_ARG, "zero quaternion");
            double w = q[0] / nq, x = q[1] / nq, y = q[2] / nq, z = q[3] / nq;
            Rot9 R{{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                    2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                    2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
            k_rotate_template<<<64, 256, 0, st>>>(tp.as<double>(), tz, ty, tx, R, 1.0 / (double)V, rot.as<float>());
            TTM_LAUNCH_CHECK();
            launch_r2c_any<float>(SrcTemplateRows{rot.as<float>(), Y, X, ty, tx}, (int64_t)tz * Y, pt, p.px32, st);
            launch_strided_any<float, -1>(pt, StridedAxis{Xh, tz, ncols, Xh}, p.py32, ProIdentity<float>(),
                                      StoreTo<float>{pt, ncols, Xh}, st);
            const DeviceWait dw = ctx->wait();
            launch_zcorr(p.G.as<float2>(), pt, 1, tz, tz / 2, ncols, wk, p.pz32, (const float*)nullptr, 1.f, st, &dw);
            launch_strided_any<float, +1>(wk, StridedAxis{Xh, Z, ncols, Xh}, p.py32, ProIdentity<float>(),
                                      StoreTo<float>{wk, ncols, Xh}, st);
            launch_c2r_any<float>(wk, (int64_t)Z * Y, SinkTMMax{p.w.as<float>(), d_best, d_best_idx, X, (int32_t)j},
                                   p.px32, 1, st);
        }
        TTM_CUDA_TRY(cudaStreamSynchronize(st));
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(ctx, e);
    }
}
