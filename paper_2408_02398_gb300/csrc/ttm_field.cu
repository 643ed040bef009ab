// ttm_field.cu -- the tensorial template (Eq. 9, Alg. 1) in FP64 on the GPU,
// and the template normalisation of Eq. 4 that precedes it.
//
//   t' = m (S(t) - mu) / sqrt(<S(t)^2,1> - <S(t),1>^2 / M),  S(t) = m (h * t)
//   T_alpha(p) = (1/|Q|) sum_q u_q^alpha t'(R_q^T p),
//   u_q = R_q e_z (d' = 3) or u_q = q itself (d' = 4, the quaternion form)
//
// The field kernel gives every thread one template voxel p and streams the
// rotations through shared memory in chunks (rotation matrix and the K
// monomial weights of each q, precomputed on the host); t'(R^T p) is a
// trilinear sample. Voxels farther than r + soft + sqrt(3) from the centre
// get no contribution (every trilinear neighbour is outside the mask) and
// are written as exact zeros.
#include <cmath>
#include <vector>

#include "ttm_internal.h"

namespace ttm {

// Eq. 4 on the template grid, one CTA: S = m (h * t) in FP64, the three
// sums, then t'. tmp holds S.
__global__ void __launch_bounds__(1024)
k_normalise_template(const float* __restrict__ t, const double* __restrict__ m, int tz, int ty, int tx, double a,
                     double* __restrict__ S, double* __restrict__ tp, double* __restrict__ stats)
{
    __shared__ double r_sm[1024], r_s[1024], r_s2[1024], r_m[1024];
    const int n = tz * ty * tx;
    const double tap[3] = {a, 1.0 - 2.0 * a, a};
    double sm = 0, s1 = 0, s2 = 0, mm = 0;
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
        int x = v % tx, y = (v / tx) % ty, z = v / (tx * ty);
        double h = 0;
        for (int dz = -1; dz <= 1; dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    int zz = z + dz, yy = y + dy, xx = x + dx;
                    if (zz < 0 || zz >= tz || yy < 0 || yy >= ty || xx < 0 || xx >= tx) continue;
                    h += tap[dz + 1] * tap[dy + 1] * tap[dx + 1] * (double)t[(zz * ty + yy) * tx + xx];
                }
        double sv = m[v] * h;
        S[v] = sv;
        sm += sv * m[v];
        s1 += sv;
        s2 += sv * sv;
        mm += m[v];
    }
    r_sm[threadIdx.x] = sm; r_s[threadIdx.x] = s1; r_s2[threadIdx.x] = s2; r_m[threadIdx.x] = mm;
    __syncthreads();
    for (int hh = blockDim.x / 2; hh > 0; hh >>= 1) {
        if (threadIdx.x < hh) {
            r_sm[threadIdx.x] += r_sm[threadIdx.x + hh];
            r_s[threadIdx.x] += r_s[threadIdx.x + hh];
            r_s2[threadIdx.x] += r_s2[threadIdx.x + hh];
            r_m[threadIdx.x] += r_m[threadIdx.x + hh];
        }
        __syncthreads();
    }
    const double M = r_m[0];
    const double mu = r_sm[0] / M;
    const double den = sqrt(r_s2[0] - r_s[0] * r_s[0] / M);
    if (threadIdx.x == 0) { stats[0] = mu; stats[1] = den; stats[2] = M; }
    for (int v = threadIdx.x; v < n; v += blockDim.x) tp[v] = den > 0 ? m[v] * (S[v] - mu) / den : 0.0;
}

__device__ __forceinline__ double trilinear64(const double* __restrict__ v, int tz, int ty, int tx, double fx,
                                              double fy, double fz)
{
    double x0 = floor(fx), y0 = floor(fy), z0 = floor(fz);
    double ax = fx - x0, ay = fy - y0, az = fz - z0;
    int ix = (int)x0, iy = (int)y0, iz = (int)z0;
    double acc = 0;
#pragma unroll
    for (int dz = 0; dz <= 1; dz++)
#pragma unroll
        for (int dy = 0; dy <= 1; dy++)
#pragma unroll
            for (int dx = 0; dx <= 1; dx++) {
                int xx = ix + dx, yy = iy + dy, zz = iz + dz;
                if (xx < 0 || xx >= tx || yy < 0 || yy >= ty || zz < 0 || zz >= tz) continue;
                double wgt = (dx ? ax : 1 - ax) * (dy ? ay : 1 - ay) * (dz ? az : 1 - az);
                acc += wgt * v[((int64_t)zz * ty + yy) * tx + xx];
            }
    return acc;
}

constexpr int kFieldThreads = 128;
constexpr int kFieldChunk = 32;

// qdata: per rotation 9 entries of R (row-major) then the weights u^alpha
// of the K components [k0, k0 + K) of this launch (the host splits a large
// component count into several launches); T points at component k0.
template <int K>
__global__ void __launch_bounds__(kFieldThreads)
k_field(const double* __restrict__ tp, int tz, int ty, int tx, const double* __restrict__ qdata, int64_t nq,
        double rmax2, double inv_nq, double* __restrict__ T)
{
    constexpr int QS = 9 + K;
    __shared__ double qs[kFieldChunk * QS];
    const int n = tz * ty * tx;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    const int cz = tz / 2, cy = ty / 2, cx = tx / 2;
    int x = 0, y = 0, z = 0;
    if (v < n) { x = v % tx; y = (v / tx) % ty; z = v / (tx * ty); }
    const double px = x - cx, py = y - cy, pz = z - cz;
    const bool active = v < n && (px * px + py * py + pz * pz) <= rmax2;
    // a whole CTA can be outside the support: then it only writes zeros
    const bool any = __syncthreads_or(active);
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; k++) acc[k] = 0.0;
    if (any) {
        for (int64_t q0 = 0; q0 < nq; q0 += kFieldChunk) {
            const int nc = (int)min((int64_t)kFieldChunk, nq - q0);
            __syncthreads();
            for (int i = threadIdx.x; i < nc * QS; i += blockDim.x) qs[i] = qdata[q0 * QS + i];
            __syncthreads();
            if (!active) continue;
            for (int c = 0; c < nc; c++) {
                const double* R = qs + c * QS;
                // R^T p
                double sx = R[0] * px + R[3] * py + R[6] * pz;
                double sy = R[1] * px + R[4] * py + R[7] * pz;
                double sz = R[2] * px + R[5] * py + R[8] * pz;
                double val = trilinear64(tp, tz, ty, tx, sx + cx, sy + cy, sz + cz);
                if (val == 0.0) continue;
                const double* wq = R + 9;
#pragma unroll
                for (int k = 0; k < K; k++) acc[k] += wq[k] * val;
            }
        }
    }
    if (v < n) {
#pragma unroll
        for (int k = 0; k < K; k++) T[(int64_t)k * n + v] = acc[k] * inv_nq;
    }
}

// ---------------------------------------------------------------- host --

// super-Fibonacci spiral samples of SO(3) (Alexa, CVPR 2022): for
// s = i + 1/2, (sqrt(s/N) sin a, sqrt(s/N) cos a, sqrt(1-s/N) sin b,
// sqrt(1-s/N) cos b) with a = 2 pi s / sqrt(2), b = 2 pi s / psi and psi the
// real root of psi^4 = psi + 4; the four entries are (w, x, y, z).
static double psi_root()
{
    // bisection on f(x) = x^4 - x - 4 over [1, 2]
    double lo = 1.0, hi = 2.0;
    for (int i = 0; i < 200; i++) {
        double mid = 0.5 * (lo + hi);
        double f = mid * mid * mid * mid - mid - 4.0;
        (f > 0 ? hi : lo) = mid;
    }
    return 0.5 * (lo + hi);
}

static void quat_mul(const double* a, const double* b, double* o)
{
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

static void rot_of(const double* q, double* R)
{
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

// the 24 rotations of the cube from the signed permutation matrices of
// determinant +1, converted to unit quaternions with w >= 0
static std::vector<double> cube_quaternions()
{
    std::vector<double> out;
    const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (auto& pm : perms)
        for (int sgn = 0; sgn < 8; sgn++) {
            double P[9] = {0};
            for (int r = 0; r < 3; r++) P[r * 3 + pm[r]] = (sgn >> r) & 1 ? -1.0 : 1.0;
            double det = P[0] * (P[4] * P[8] - P[5] * P[7]) - P[1] * (P[3] * P[8] - P[5] * P[6]) +
                         P[2] * (P[3] * P[7] - P[4] * P[6]);
            if (det < 0) continue;
            // matrix -> quaternion (branch on the largest diagonal combination)
            double tr = P[0] + P[4] + P[8];
            double q[4];
            if (tr > 0) {
                double s = std::sqrt(tr + 1.0) * 2;
                q[0] = 0.25 * s; q[1] = (P[7] - P[5]) / s; q[2] = (P[2] - P[6]) / s; q[3] = (P[3] - P[1]) / s;
            } else if (P[0] > P[4] && P[0] > P[8]) {
                double s = std::sqrt(1.0 + P[0] - P[4] - P[8]) * 2;
                q[0] = (P[7] - P[5]) / s; q[1] = 0.25 * s; q[2] = (P[1] + P[3]) / s; q[3] = (P[2] + P[6]) / s;
            } else if (P[4] > P[8]) {
                double s = std::sqrt(1.0 + P[4] - P[0] - P[8]) * 2;
                q[0] = (P[2] - P[6]) / s; q[1] = (P[1] + P[3]) / s; q[2] = 0.25 * s; q[3] = (P[5] + P[7]) / s;
            } else {
                double s = std::sqrt(1.0 + P[8] - P[0] - P[4]) * 2;
                q[0] = (P[3] - P[1]) / s; q[1] = (P[2] + P[6]) / s; q[2] = (P[5] + P[7]) / s; q[3] = 0.25 * s;
            }
            if (q[0] < 0) for (double& c : q) c = -c;
            out.insert(out.end(), q, q + 4);
        }
    return out;
}

void rotation_set(int64_t n_base, bool cube, std::vector<double>& q)
{
    const double phi = std::sqrt(2.0), psi = psi_root();
    std::vector<double> base(4 * n_base);
    for (int64_t i = 0; i < n_base; i++) {
        double s = (double)i + 0.5;
        double r = std::sqrt(s / (double)n_base), R = std::sqrt(1.0 - s / (double)n_base);
        double al = 2.0 * M_PI * s / phi, be = 2.0 * M_PI * s / psi;
        base[4 * i + 0] = r * std::sin(al);
        base[4 * i + 1] = r * std::cos(al);
        base[4 * i + 2] = R * std::sin(be);
        base[4 * i + 3] = R * std::cos(be);
    }
    if (!cube) { q.swap(base); return; }
    std::vector<double> c = cube_quaternions();
    q.assign(4 * n_base * 24, 0.0);
    for (int64_t i = 0; i < n_base; i++)
        for (int j = 0; j < 24; j++) quat_mul(&c[4 * j], &base[4 * i], &q[4 * (i * 24 + j)]);
}

// graded-lex descending exponents (a, b, c) of (x, y, z) with a+b+c = n
void exponents3(int n, std::vector<int>& e)
{
    e.clear();
    for (int a = n; a >= 0; a--)
        for (int b = n - a; b >= 0; b--) { e.push_back(a); e.push_back(b); e.push_back(n - a - b); }
}

// the same order for (w, x, y, z): exponents (a, b, c, d), a+b+c+d = n
void exponents4(int n, std::vector<int>& e)
{
    e.clear();
    for (int a = n; a >= 0; a--)
        for (int b = n - a; b >= 0; b--)
            for (int c = n - a - b; c >= 0; c--) {
                e.push_back(a); e.push_back(b); e.push_back(c); e.push_back(n - a - b - c);
            }
}

// device t' (FP64) of a raw float template under params; returns in tp
void normalise_template_dev(ttm_ctx* ctx, const float* d_tmpl, int tz, int ty, int tx,
                            const ttm_field_params& fp, DevBuf& tp, cudaStream_t st)
{
    (void)ctx;
    std::vector<double> m;
    double M = make_mask(tz, ty, tx, fp.mask_radius, fp.mask_soft_width, m);
    TTM_REQUIRE(M > 0, E_INVALID_ARG, "mask is empty");
    const size_t n = (size_t)tz * ty * tx;
    DevBuf dm, S, stats;
    dm.alloc(n * sizeof(double));
    S.alloc(n * sizeof(double));
    stats.alloc(4 * sizeof(double));
    tp.alloc(n * sizeof(double));
    TTM_CUDA_TRY(cudaMemcpyAsync(dm.p, m.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    k_normalise_template<<<1, 1024, 0, st>>>(d_tmpl, dm.as<double>(), tz, ty, tx, fp.filter_a, S.as<double>(),
                                             tp.as<double>(), stats.as<double>());
    TTM_LAUNCH_CHECK();
    TTM_CUDA_TRY(cudaStreamSynchronize(st));
}

}  // namespace ttm

using namespace ttm;

extern "C" ttm_status ttm_rotation_set(int64_t n_base, int cube, double* h_quats)
{
    if (n_base <= 0 || !h_quats) return TTM_E_INVALID_ARG;
    std::vector<double> q;
    rotation_set(n_base, cube != 0, q);
    std::copy(q.begin(), q.end(), h_quats);
    return TTM_OK;
}

extern "C" ttm_status ttm_build_tensor_field(ttm_ctx* ctx, const float* d_tmpl, int tz, int ty, int tx,
                                             const ttm_field_params* params, double* d_field, void* stream)
{
    if (!ctx) return TTM_E_INVALID_ARG;
    try {
        TTM_REQUIRE(d_tmpl && d_field && params, E_INVALID_ARG, "null pointer argument");
        TTM_REQUIRE(tz > 0 && ty > 0 && tx > 0, E_SHAPE, "bad template shape");
        TTM_REQUIRE(params->order_n == 2 || params->order_n == 4 || params->order_n == 6, E_UNSUPPORTED,
                    "order_n must be 2, 4 or 6");
        TTM_REQUIRE(params->dprime == 3 || params->dprime == 4, E_INVALID_ARG, "dprime must be 3 or 4");
        TTM_REQUIRE(params->n_rot_base > 0, E_INVALID_ARG, "n_rot_base must be positive");
        TTM_REQUIRE(params->mask_radius > 0 && params->filter_a >= 0 && params->filter_a < 0.25, E_INVALID_ARG,
                    "bad mask radius or filter parameter");
        TTM_CUDA_TRY(cudaSetDevice(ctx->device));
        cudaStream_t st = (cudaStream_t)stream;
        DevBuf tp;
        normalise_template_dev(ctx, d_tmpl, tz, ty, tx, *params, tp, st);

        const int n = params->order_n;
        const int dp = params->dprime;
        std::vector<double> quats;
        rotation_set(params->n_rot_base, params->cube_symmetrize != 0, quats);
        const int64_t nq = (int64_t)quats.size() / 4;
        std::vector<int> e;
        if (dp == 3) exponents3(n, e); else exponents4(n, e);
        const int K = (int)e.size() / dp;
        // components per launch: all of them up to 35, else chunks of 28
        // (the per-thread FP64 accumulators stay in registers)
        const int KC = K <= 35 ? K : 28;
        TTM_REQUIRE(K % KC == 0, E_UNSUPPORTED, "unsupported component count");
        const int QS = 9 + KC;
        const double rmax = params->mask_radius + params->mask_soft_width + std::sqrt(3.0) + 1e-9;
        const int nvox = tz * ty * tx;
        const int grid = (int)ceil_div(nvox, kFieldThreads);
        const double inv = 1.0 / (double)nq;
        std::vector<double> qd((size_t)nq * QS);
        DevBuf dq;
        dq.alloc(qd.size() * sizeof(double));
        for (int k0 = 0; k0 < K; k0 += KC) {
            for (int64_t i = 0; i < nq; i++) {
                double* R = &qd[(size_t)i * QS];
                const double* q = &quats[4 * i];
                rot_of(q, R);
                double u[4];
                if (dp == 3) { u[0] = R[2]; u[1] = R[5]; u[2] = R[8]; }  // R e_z
                else { u[0] = q[0]; u[1] = q[1]; u[2] = q[2]; u[3] = q[3]; }
                for (int k = 0; k < KC; k++) {
                    double wgt = 1.0;
                    for (int d = 0; d < dp; d++)
                        for (int p = 0; p < e[dp * (k0 + k) + d]; p++) wgt *= u[d];
                    R[9 + k] = wgt;
                }
            }
            // the previous launch reads dq: copy in stream order
            TTM_CUDA_TRY(cudaMemcpyAsync(dq.p, qd.data(), qd.size() * sizeof(double), cudaMemcpyHostToDevice, st));
            double* Tk = d_field + (size_t)k0 * nvox;
            switch (KC) {
                case 6: k_field<6><<<grid, kFieldThreads, 0, st>>>(tp.as<double>(), tz, ty, tx, dq.as<double>(), nq, rmax * rmax, inv, Tk); break;
                case 10: k_field<10><<<grid, kFieldThreads, 0, st>>>(tp.as<double>(), tz, ty, tx, dq.as<double>(), nq, rmax * rmax, inv, Tk); break;
                case 15: k_field<15><<<grid, kFieldThreads, 0, st>>>(tp.as<double>(), tz, ty, tx, dq.as<double>(), nq, rmax * rmax, inv, Tk); break;
                case 28: k_field<28><<<grid, kFieldThreads, 0, st>>>(tp.as<double>(), tz, ty, tx, dq.as<double>(), nq, rmax * rmax, inv, Tk); break;
                case 35: k_field<35><<<grid, kFieldThreads, 0, st>>>(tp.as<double>(), tz, ty, tx, dq.as<double>(), nq, rmax * rmax, inv, Tk); break;
                default: throw Error{E_UNSUPPORTED, "unsupported component count"};
            }
            TTM_LAUNCH_CHECK();
            // qd is rewritten for the next chunk: the copy above must be done
            if (k0 + KC < K) TTM_CUDA_TRY(cudaStreamSynchronize(st));
        }
        // tp and dq are freed on return: wait for the kernel that reads them
        TTM_CUDA_TRY(cudaStreamSynchronize(st));
        return TTM_OK;
    } catch (const Error& e) {
        return (ttm_status)fail(ctx, e);
    }
}
