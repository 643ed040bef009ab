// ttm_refine.cu -- position refinement of TTM peaks (TTM-ref, Sec. 3.3 and
// Alg. 3). For each peak x_i the voxels of the ball ||x - x_i|| <= r_s are
// scored by the LNCC at their own optimal rotation,
//   c(x) = w(x) sum_z t'(R(q*(x))^T z) g(x + z),
// in real space (the template window around x, trilinear samples of the
// normalised template t', zero outside its grid), and the peak moves to the
// best of them. q*(x) is the quaternion map of the d' = 4 maximiser; g and
// w are the filtered tomogram and local normaliser of the plan's last
// correlation (Eq. 2, Eq. 3).
//
// One CTA per (peak, candidate): its threads stride over the template
// voxels with FP32 samples and partial sums, reduced in FP64. The
// candidates of a peak are the peak itself, then the other ball voxels in
// (z, y, x) order; the host keeps the first strictly higher LNCC in that
// order (Alg. 3). Candidates outside the valid box (whose template window
// leaves the tomogram) are not scored.
#include <cmath>
#include <vector>

#include "ttm_internal.h"

namespace ttm {

constexpr int kRefThreads = 256;

struct RefGeom {
    int Z, Y, X;                 // working grid of g and w
    int b[6];                    // valid box (z0, z1, y0, y1, x0, x1)
    int tz, ty, tx;              // template grid
    int64_t V;                   // Z * Y * X (component stride of the quaternion map)
};

__device__ __forceinline__ float trilinear32(const float* __restrict__ v, int tz, int ty, int tx, float fx, float fy,
                                             float fz)
{
    const float x0 = floorf(fx), y0 = floorf(fy), z0 = floorf(fz);
    const float ax = fx - x0, ay = fy - y0, az = fz - z0;
    const int ix = (int)x0, iy = (int)y0, iz = (int)z0;
    float acc = 0.f;
#pragma unroll
    for (int dz = 0; dz <= 1; dz++)
#pragma unroll
        for (int dy = 0; dy <= 1; dy++)
#pragma unroll
            for (int dx = 0; dx <= 1; dx++) {
                const int xx = ix + dx, yy = iy + dy, zz = iz + dz;
                if (xx < 0 || xx >= tx || yy < 0 || yy >= ty || zz < 0 || zz >= tz) continue;
                const float wgt = (dx ? ax : 1.f - ax) * (dy ? ay : 1.f - ay) * (dz ? az : 1.f - az);
                acc += wgt * __ldg(v + ((int64_t)zz * ty + yy) * tx + xx);
            }
    return acc;
}

// grid (n_cand, P): candidate j of peak i; writes the LNCC (or -inf outside
// the valid box) and the candidate's quaternion
__global__ void __launch_bounds__(kRefThreads)
k_refine_lncc(const float* __restrict__ g, const float* __restrict__ w, const float* __restrict__ orient,
              const float* __restrict__ tp, const int64_t* __restrict__ peaks, const int* __restrict__ offs,
              int n_cand, RefGeom geo, double* __restrict__ c_out, float* __restrict__ q_out)
{
    __shared__ double red[kRefThreads / 32];
    const int j = blockIdx.x, i = blockIdx.y;
    const int64_t pk = peaks[i];
    const int px = (int)(pk % geo.X), py = (int)((pk / geo.X) % geo.Y), pz = (int)(pk / ((int64_t)geo.X * geo.Y));
    const int z = pz + offs[3 * j], y = py + offs[3 * j + 1], x = px + offs[3 * j + 2];
    const int64_t slot = (int64_t)i * n_cand + j;
    const bool inside = z >= geo.b[0] && z < geo.b[1] && y >= geo.b[2] && y < geo.b[3] && x >= geo.b[4] && x < geo.b[5];
    if (!inside) {  // uniform over the CTA
        if (threadIdx.x == 0) {
            c_out[slot] = -INFINITY;
            for (int k = 0; k < 4; k++) q_out[4 * slot + k] = 0.f;
        }
        return;
    }
    const int64_t v = ((int64_t)z * geo.Y + y) * geo.X + x;
    const float qw = orient[v], qx = orient[geo.V + v], qy = orient[2 * geo.V + v], qz = orient[3 * geo.V + v];
    // R(q), row-major, acting on (x, y, z) column vectors
    const float R0 = 1.f - 2.f * (qy * qy + qz * qz), R1 = 2.f * (qx * qy - qw * qz), R2 = 2.f * (qx * qz + qw * qy);
    const float R3 = 2.f * (qx * qy + qw * qz), R4 = 1.f - 2.f * (qx * qx + qz * qz), R5 = 2.f * (qy * qz - qw * qx);
    const float R6 = 2.f * (qx * qz - qw * qy), R7 = 2.f * (qy * qz + qw * qx), R8 = 1.f - 2.f * (qx * qx + qy * qy);
    const int cz = geo.tz / 2, cy = geo.ty / 2, cx = geo.tx / 2;
    const int nt = geo.tz * geo.ty * geo.tx;
    float acc = 0.f;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        const int tx_ = t % geo.tx, ty_ = (t / geo.tx) % geo.ty, tz_ = t / (geo.tx * geo.ty);
        const float ox = (float)(tx_ - cx), oy = (float)(ty_ - cy), oz = (float)(tz_ - cz);
        // t'_R(o) = t'(R^T o)
        const float sx = R0 * ox + R3 * oy + R6 * oz, sy = R1 * ox + R4 * oy + R7 * oz,
                    sz = R2 * ox + R5 * oy + R8 * oz;
        const float tv = trilinear32(tp, geo.tz, geo.ty, geo.tx, sx + cx, sy + cy, sz + cz);
        if (tv != 0.f) acc += tv * __ldg(g + ((int64_t)(z + tz_ - cz) * geo.Y + (y + ty_ - cy)) * geo.X + (x + tx_ - cx));
    }
    double d = acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < kRefThreads / 32; k++) s += red[k];
        c_out[slot] = (double)w[v] * s;
        q_out[4 * slot] = qw; q_out[4 * slot + 1] = qx; q_out[4 * slot + 2] = qy; q_out[4 * slot + 3] = qz;
    }
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = (float)a[i];
}

// Alg. 3's candidate set: the peak, then the rest of the ball in (z, y, x) order
static std::vector<int> ball_offsets(double rs)
{
    std::vector<int> o = {0, 0, 0};
    const int R = (int)std::floor(rs);
    for (int dz = -R; dz <= R; dz++)
        for (int dy = -R; dy <= R; dy++)
            for (int dx = -R; dx <= R; dx++) {
                if (dz == 0 && dy == 0 && dx == 0) continue;
                if ((double)(dz * dz + dy * dy + dx * dx) > rs * rs) continue;
                o.push_back(dz); o.push_back(dy); o.push_back(dx);
            }
    return o;
}

}  // namespace ttm

using namespace ttm;

extern "C" ttm_status ttm_refine_peaks(ttm_plan* plan, const float* d_tmpl, const float* d_orient,
                                       const int64_t* h_peaks, int P, double r_s, int64_t* h_idx, float* h_quat,
                                       float* h_lncc, void* stream)
{
    if (!plan) return TTM_E_INVALID_ARG;
    try {
        TTM_REQUIRE(d_tmpl && d_orient && (P == 0 || (h_peaks && h_idx && h_quat && h_lncc)), E_INVALID_ARG,
                    "null pointer argument");
        TTM_REQUIRE(plan->fp.dprime == 4, E_UNSUPPORTED, "refinement needs the rotation map of the d' = 4 form");
        TTM_REQUIRE(P >= 0 && P <= 65535 && r_s >= 0 && r_s <= 16, E_INVALID_ARG,
                    "P must be in [0, 65535] and r_s in [0, 16]");
        if (P == 0) return TTM_OK;
        TTM_CUDA_TRY(cudaSetDevice(plan->ctx->device));
        cudaStream_t st = (cudaStream_t)stream;
        const Prep& p = plan->prep;
        RefGeom geo;
        geo.Z = p.Z; geo.Y = p.Y; geo.X = p.X;
        ttm_plan_valid_box(plan, geo.b);
        geo.tz = p.tz; geo.ty = p.ty; geo.tx = p.tx;
        geo.V = (int64_t)p.Z * p.Y * p.X;
        for (int i = 0; i < P; i++) {
            const int64_t v = h_peaks[i];
            TTM_REQUIRE(v >= 0 && v < geo.V, E_INVALID_ARG, "peak index outside the grid");
            const int x = (int)(v % p.X), y = (int)((v / p.X) % p.Y), z = (int)(v / ((int64_t)p.X * p.Y));
            TTM_REQUIRE(z >= geo.b[0] && z < geo.b[1] && y >= geo.b[2] && y < geo.b[3] && x >= geo.b[4] &&
                            x < geo.b[5],
                        E_INVALID_ARG, "peak outside the valid box");
        }
        // t' in FP32 (Eq. 4, the same normalisation as the tensor field)
        DevBuf tp64, tp32;
        normalise_template_dev(plan->ctx, d_tmpl, p.tz, p.ty, p.tx, plan->fp, tp64, st);
        const int nt = p.tz * p.ty * p.tx;
        tp32.alloc((size_t)nt * sizeof(float));
        k_to_float<<<(unsigned)std::min<int64_t>(1024, ceil_div(nt, 256)), 256, 0, st>>>(tp64.as<double>(),
                                                                                          tp32.as<float>(), nt);
        TTM_LAUNCH_CHECK();
        const std::vector<int> offs = ball_offsets(r_s);
        const int n_cand = (int)offs.size() / 3;
        DevBuf d_offs, d_peaks, d_c, d_q;
        d_offs.alloc(offs.size() * sizeof(int));
        d_peaks.alloc((size_t)P * sizeof(int64_t));
        d_c.alloc((size_t)P * n_cand * sizeof(double));
        d_q.alloc((size_t)P * n_cand * 4 * sizeof(float));
        TTM_CUDA_TRY(cudaMemcpyAsync(d_offs.p, offs.data(), offs.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        TTM_CUDA_TRY(cudaMemcpyAsync(d_peaks.p, h_peaks, (size_t)P * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        k_refine_lncc<<<dim3((unsigned)n_cand, (unsigned)P), kRefThreads, 0, st>>>(
            p.g32.as<float>(), p.w.as<float>(), d_orient, tp32.as<float>(), d_peaks.as<int64_t>(), d_offs.as<int>(),
            n_cand, geo, d_c.as<double>(), d_q.as<float>());
        TTM_LAUNCH_CHECK();
        std::vector<double> c((size_t)P * n_cand);
        std::vector<float> q((size_t)P * n_cand * 4);
        TTM_CUDA_TRY(cudaMemcpyAsync(c.data(), d_c.p, c.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        TTM_CUDA_TRY(cudaMemcpyAsync(q.data(), d_q.p, q.size() * sizeof(float), cudaMemcpyDeviceToHost, st));
        TTM_CUDA_TRY(cudaStreamSynchronize(st));
        for (int i = 0; i < P; i++) {
            int best = 0;  // the peak itself (inside the valid box, so scored)
            for (int j = 1; j < n_cand; j++)
                if (c[(size_t)i * n_cand + j] > c[(size_t)i * n_cand + best]) best = j;
            const int64_t v = h_peaks[i];
            const int x = (int)(v % p.X), y = (int)((v / p.X) % p.Y), z = (int)(v / ((int64_t)p.X * p.Y));
            h_idx[i] = ((int64_t)(z + offs[3 * best]) * p.Y + (y + offs[3 * best + 1])) * p.X + (x + offs[3 * best + 2]);
            for (int k = 0; k < 4; k++) h_quat[4 * i + k] = q[((size_t)i * n_cand + best) * 4 + k];
            h_lncc[i] = (float)c[(size_t)i * n_cand + best];
        }
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(plan->ctx, e);
    }
}
