// mlp_mma.cuh -- inference of the warm-start MLP (K -> 128 -> 128 -> 3,
// GELU in its tanh form) for the 32 rows held by one warp, on the tensor
// cores with mma.sync m16n8k16 (BF16 operands, FP32 accumulation).
//
// Shared-memory image (BF16 rows padded so that the fragment loads of the
// eight row groups of a warp fall into distinct banks):
//   W1 [128][kW1S]  (input columns 0..KX-1, zero beyond K)
//   W2 [128][kW2S]
//   W3 [8][kW2S]    (rows 3..7 zero)
//   b1 [128], b2 [128], b3 [4] FP32
// The same image, byte for byte, is kept in device memory by the MLP
// object and copied into shared memory by the kernels that use it.
//
// Fragment layouts of m16n8k16 (lane = 4 * g + t): A (row-major 16 x 16)
// a0 = (g, 2t..2t+1), a1 = (g+8, 2t..), a2 = (g, 2t+8..), a3 = (g+8, 2t+8..);
// B (16 x 8, k-major per column) b0 = (k 2t..2t+1, n g), b1 = (k 2t+8.., n g);
// C c0, c1 = (g, 2t..2t+1), c2, c3 = (g+8, 2t..2t+1). The accumulators of
// two adjacent 8-column tiles are therefore exactly the A fragment of the
// next layer's 16-wide k step, so the hidden activations never leave
// registers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>

namespace ttm {

constexpr int kMlpH = 128;
constexpr int kW1S = 40;   // BF16 row stride of W1 and of the staged inputs
constexpr int kW2S = 136;  // BF16 row stride of W2 and W3
constexpr size_t kMlpOffW1 = 0;
constexpr size_t kMlpOffW2 = kMlpOffW1 + sizeof(__nv_bfloat16) * kMlpH * kW1S;
constexpr size_t kMlpOffW3 = kMlpOffW2 + sizeof(__nv_bfloat16) * kMlpH * kW2S;
constexpr size_t kMlpOffB1 = kMlpOffW3 + sizeof(__nv_bfloat16) * 8 * kW2S;
constexpr size_t kMlpOffB2 = kMlpOffB1 + sizeof(float) * kMlpH;
constexpr size_t kMlpOffB3 = kMlpOffB2 + sizeof(float) * kMlpH;
constexpr size_t kMlpImageBytes = kMlpOffB3 + sizeof(float) * 4;  // 48,272
static_assert(kMlpImageBytes % 16 == 0, "image is copied in 16-byte units");

__host__ __device__ constexpr int mlp_kx(int K) { return (K + 15) / 16 * 16; }

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// the same shape with FP16 operands
__device__ __forceinline__ void mma_f16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t ld_b32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float gelu_fast(float x)
{
    const float c = 0.7978845608028654f;  // sqrt(2 / pi)
    return 0.5f * x * (1.f + tanh_approx(c * (x + 0.044715f * x * x * x)));
}

// copy the parameter image into shared memory (all threads of the CTA)
__device__ __forceinline__ void mlp_image_to_smem(const unsigned char* __restrict__ g, unsigned char* s)
{
    const uint4* src = reinterpret_cast<const uint4*>(g);
    uint4* dst = reinterpret_cast<uint4*>(s);
    for (int i = threadIdx.x; i < (int)(kMlpImageBytes / 16); i += blockDim.x) dst[i] = src[i];
}

// The warp's 32 input rows are in sx [32][kW1S] (BF16, columns >= K zero);
// the pre-bias outputs y go to sy [32][4] (columns 0..2).
template <int KX>
__device__ __forceinline__ void mlp_warp_bf16(const __nv_bfloat16* sx, const unsigned char* img, float* sy)
{
    const __nv_bfloat16* W1 = reinterpret_cast<const __nv_bfloat16*>(img + kMlpOffW1);
    const __nv_bfloat16* W2 = reinterpret_cast<const __nv_bfloat16*>(img + kMlpOffW2);
    const __nv_bfloat16* W3 = reinterpret_cast<const __nv_bfloat16*>(img + kMlpOffW3);
    const float* b1 = reinterpret_cast<const float*>(img + kMlpOffB1);
    const float* b2 = reinterpret_cast<const float*>(img + kMlpOffB2);
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll 1
    for (int mt = 0; mt < 2; mt++) {
        const int r0 = 16 * mt + g, r1 = r0 + 8;
        uint32_t a1[KX / 16][4];
#pragma unroll
        for (int ks = 0; ks < KX / 16; ks++) {
            a1[ks][0] = ld_b32(sx + r0 * kW1S + 16 * ks + 2 * t);
            a1[ks][1] = ld_b32(sx + r1 * kW1S + 16 * ks + 2 * t);
            a1[ks][2] = ld_b32(sx + r0 * kW1S + 16 * ks + 8 + 2 * t);
            a1[ks][3] = ld_b32(sx + r1 * kW1S + 16 * ks + 8 + 2 * t);
        }
        // layer 1 -> bias -> GELU, packed straight into layer-2 A fragments
        uint32_t a2[8][4];
#pragma unroll
        for (int nt = 0; nt < 16; nt++) {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            const __nv_bfloat16* wr = W1 + (nt * 8 + g) * kW1S + 2 * t;
#pragma unroll
            for (int ks = 0; ks < KX / 16; ks++) mma_bf16(acc, a1[ks], ld_b32(wr + 16 * ks), ld_b32(wr + 16 * ks + 8));
            const int j = nt * 8 + 2 * t;
            const float h0 = gelu_fast(acc[0] + b1[j]), h1 = gelu_fast(acc[1] + b1[j + 1]);
            const float h2 = gelu_fast(acc[2] + b1[j]), h3 = gelu_fast(acc[3] + b1[j + 1]);
            a2[nt >> 1][(nt & 1) * 2] = pack_bf16(h0, h1);
            a2[nt >> 1][(nt & 1) * 2 + 1] = pack_bf16(h2, h3);
        }
        // layer 2 in pairs of 8-column tiles, each pair feeding one k step
        // of layer 3
        float y[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks3 = 0; ks3 < 8; ks3++) {
            uint32_t a3[4];
#pragma unroll
            for (int half = 0; half < 2; half++) {
                const int nt = 2 * ks3 + half;
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
                const __nv_bfloat16* wr = W2 + (nt * 8 + g) * kW2S + 2 * t;
#pragma unroll
                for (int ks = 0; ks < 8; ks++) mma_bf16(acc, a2[ks], ld_b32(wr + 16 * ks), ld_b32(wr + 16 * ks + 8));
                const int j = nt * 8 + 2 * t;
                a3[half * 2] = pack_bf16(gelu_fast(acc[0] + b2[j]), gelu_fast(acc[1] + b2[j + 1]));
                a3[half * 2 + 1] = pack_bf16(gelu_fast(acc[2] + b2[j]), gelu_fast(acc[3] + b2[j + 1]));
            }
            const __nv_bfloat16* wr = W3 + g * kW2S + 16 * ks3 + 2 * t;
            mma_bf16(y, a3, ld_b32(wr), ld_b32(wr + 8));
        }
        if (t == 0) {
            sy[r0 * 4 + 0] = y[0]; sy[r0 * 4 + 1] = y[1];
            sy[r1 * 4 + 0] = y[2]; sy[r1 * 4 + 1] = y[3];
        } else if (t == 1) {
            sy[r0 * 4 + 2] = y[0];
            sy[r1 * 4 + 2] = y[2];
        }
    }
}

}  // namespace ttm
