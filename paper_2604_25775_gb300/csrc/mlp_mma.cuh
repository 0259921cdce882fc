// mlp_mma.cuh -- the site-wise layers of Eq. MLP on the tensor cores, one warp per 16-row
// tile, FP32 accumulation, activations kept in registers from layer to layer.
//
// Every product x.W is taken as three products of a two-term split, x_hi W_hi + x_lo W_hi +
// x_hi W_lo with x_hi = round(x), x_lo = round(x - x_hi) (same split of W), accumulated in
// FP32. Three input formats:
//   kTF32 (mixed mode):      TF32 (10-bit mantissa) -> about 2^-21 relative per layer,
//                            FP32-level local energies;
//   kFP16 (mixed-FP16 mode): FP16 (10-bit mantissa), k = 16 per instruction (half the MMAs
//                            of TF32); the 5-bit exponent would push the lo parts of small
//                            values into subnormals, so x enters scaled by 2^4 and each
//                            layer's W by the power of two that puts max|W| in [1/2, 1), and
//                            the FP32 accumulator is scaled back exactly: about 2^-21
//                            relative for |x| >= 2^-7, 2^-29 absolute below, and |x| must
//                            stay under 4096 (the largest FP16 / 2^4);
//   kBF16 (mixed-BF16 mode): BF16 (7-bit mantissa)  -> about 2^-16 relative per layer.
// A single BF16 product (2^-8) moves the local energies by ~1e-3 and is not offered.
//
// Fragment layouts (g = lane / 4, t = lane % 4), C (16x8, f32): c0,c1 = (g, 2t..2t+1),
// c2,c3 = (g+8, 2t..2t+1).
//   m16n8k16 bf16 / f16: A a0 = (g, 2t..2t+1), a1 = (g+8, 2t..), a2 = (g, 2t+8..), a3 = (g+8, 2t+8..)
//                  B b0 = (k 2t..2t+1, n g), b1 = (k 2t+8..2t+9, n g)
//     -> C tiles 2kk and 2kk+1 of one layer are the A fragment of k-step kk of the next.
//   m16n8k8 tf32:  A a0 = (g, t), a1 = (g+8, t), a2 = (g, t+4), a3 = (g+8, t+4)
//                  B b0 = (k t, n g), b1 = (k t+4, n g)
//     -> with the k index of each 8-wide step permuted (logical t -> channel 2t, logical
//        t+4 -> channel 2t+1, applied to W's rows as well) the C tile kk of one layer is
//        the A fragment {c0, c2, c1, c3} of k-step kk of the next.
// No shared-memory round trip is needed between layers in either format.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "scale_internal.cuh"

namespace scale {

enum MmaKind { kTF32 = 1, kBF16 = 2, kFP16 = 3 };

// kFP16: the activations enter the layer multiplied by this power of two (exact).
constexpr float kFp16InScale = 16.f;

// Per-lane weight fragments of one (layer, k-step, n-tile): {b0_hi, b1_hi, b0_lo, b1_lo}.
struct WFrag {
  uint32_t v[4];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo_k, float hi_k) {
  const __nv_bfloat162 p = __floats2bfloat162_rn(lo_k, hi_k);
  return *reinterpret_cast<const uint32_t*>(&p);
}

// x = hi + lo with hi, lo in BF16.
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
  const float ra = a - __bfloat162float(ha), rb = b - __bfloat162float(hb);
  __nv_bfloat162 h2;
  h2.x = ha;
  h2.y = hb;
  hi = *reinterpret_cast<const uint32_t*>(&h2);
  lo = pack_bf16(ra, rb);
}

// x = hi + lo with hi, lo in FP16 (the inputs already scaled into FP16's normal range).
__device__ __forceinline__ void split2h(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __half ha = __float2half_rn(a), hb = __float2half_rn(b);
  const __half2 h2 = __halves2half2(ha, hb);
  const __half2 l2 = __floats2half2_rn(a - __half2float(ha), b - __half2float(hb));
  hi = *reinterpret_cast<const uint32_t*>(&h2);
  lo = *reinterpret_cast<const uint32_t*>(&l2);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_f16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The MMA input format of a mixed precision mode.
__host__ __device__ inline int mma_kind_of(int precision) {
  return precision == SCALE_PREC_MIXED_BF16 ? kBF16 : precision == SCALE_PREC_MIXED_FP16 ? kFP16 : kTF32;
}

// Bytes of the fragment buffer of a context: sized for TF32 (L x hpad/8 k-steps x hpad/8
// n-tiles x 32 lanes).
__host__ __device__ inline size_t wfrag_bytes(int L, int hpad) {
  return (size_t)L * (hpad / 8) * (hpad / 8) * 32 * sizeof(WFrag);
}

// kFP16: the per-layer weight factors 2^-e_l ([kMaxLayers]) and output factors 2^e_l / 2^4
// ([kMaxLayers]) sit behind the fragments in the fragment buffer (FP16 fragments take half of
// it; the other half, at least 1 KB, holds the 2 x kMaxLayers factors).
__host__ __device__ inline size_t fp16_scale_offset(int L, int hpad) {
  return (size_t)L * (hpad / 16) * (hpad / 8) * 32 * sizeof(WFrag);
}
static_assert(2 * kMaxLayers * sizeof(float) <= 1 * (16 / 8) * (16 / 16) * 32 * sizeof(WFrag),
              "the FP16 scale factors fit behind the fragments of the smallest buffer");

inline float* fp16_scales(scale_ctx* c) {
  return reinterpret_cast<float*>(static_cast<char*>(c->wfrag) + fp16_scale_offset(c->L, c->hpad));
}

// Number of k-steps per layer for a format.
template <int H, int KIND>
struct MmaShape {
  static constexpr int NT = H / 8;
  static constexpr int KT = KIND == kTF32 ? H / 8 : H / 16;
};

// Layers 1..L-1 (all site-wise) on the 16-row tile held in x (C-fragment layout, FP32):
//   x <- res_l * x + act(bias_l + x W_l).
// wf: fragments [L][KT][NT][32], bias: per layer (FP32 copies); oscale (kFP16 only): per layer
// the exact factor 1 / (kFp16InScale 2^e_l) that undoes the input and weight scaling.
template <int H, int KIND>
__device__ __forceinline__ void mlp_tile(float (&x)[H / 8][4], const WFrag* __restrict__ wf,
                                         const float* const* bias, const int* resid, int L, int act,
                                         const float* __restrict__ oscale = nullptr) {
  constexpr int NT = MmaShape<H, KIND>::NT, KT = MmaShape<H, KIND>::KT;
  const int lane = threadIdx.x & 31, t = lane & 3;
  for (int l = 1; l < L; ++l) {
    uint32_t ah[KT][4], al[KT][4];
#pragma unroll
    for (int kk = 0; kk < KT; ++kk) {
      if constexpr (KIND == kTF32) {
        split_tf32(x[kk][0], ah[kk][0], al[kk][0]);
        split_tf32(x[kk][2], ah[kk][1], al[kk][1]);
        split_tf32(x[kk][1], ah[kk][2], al[kk][2]);
        split_tf32(x[kk][3], ah[kk][3], al[kk][3]);
      } else if constexpr (KIND == kFP16) {
        constexpr float S = kFp16InScale;
        split2h(S * x[2 * kk][0], S * x[2 * kk][1], ah[kk][0], al[kk][0]);
        split2h(S * x[2 * kk][2], S * x[2 * kk][3], ah[kk][1], al[kk][1]);
        split2h(S * x[2 * kk + 1][0], S * x[2 * kk + 1][1], ah[kk][2], al[kk][2]);
        split2h(S * x[2 * kk + 1][2], S * x[2 * kk + 1][3], ah[kk][3], al[kk][3]);
      } else {
        split2(x[2 * kk][0], x[2 * kk][1], ah[kk][0], al[kk][0]);
        split2(x[2 * kk][2], x[2 * kk][3], ah[kk][1], al[kk][1]);
        split2(x[2 * kk + 1][0], x[2 * kk + 1][1], ah[kk][2], al[kk][2]);
        split2(x[2 * kk + 1][2], x[2 * kk + 1][3], ah[kk][3], al[kk][3]);
      }
    }
    const WFrag* wl = wf + (size_t)l * KT * NT * 32;
    const float* bl = bias[l];
    const int res = resid[l];
    const float om = KIND == kFP16 ? oscale[l] : 1.f;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const float b0 = bl[8 * j + 2 * t], b1 = bl[8 * j + 2 * t + 1];
      // the accumulators start at the bias (kFP16: at zero, the bias added after unscaling)
      float c[4] = {b0, b1, b0, b1};
      if constexpr (KIND == kFP16) c[0] = c[1] = c[2] = c[3] = 0.f;
#pragma unroll
      for (int kk = 0; kk < KT; ++kk) {
        const WFrag w = wl[(kk * NT + j) * 32 + lane];
        if constexpr (KIND == kTF32) {
          mma_tf32(c, ah[kk], w.v[0], w.v[1]);
          mma_tf32(c, al[kk], w.v[0], w.v[1]);
          mma_tf32(c, ah[kk], w.v[2], w.v[3]);
        } else if constexpr (KIND == kFP16) {
          mma_f16(c, ah[kk], w.v[0], w.v[1]);
          mma_f16(c, al[kk], w.v[0], w.v[1]);
          mma_f16(c, ah[kk], w.v[2], w.v[3]);
        } else {
          mma_bf16(c, ah[kk], w.v[0], w.v[1]);
          mma_bf16(c, al[kk], w.v[0], w.v[1]);
          mma_bf16(c, ah[kk], w.v[2], w.v[3]);
        }
      }
      if constexpr (KIND == kFP16) {
        c[0] = fmaf(c[0], om, b0);
        c[1] = fmaf(c[1], om, b1);
        c[2] = fmaf(c[2], om, b0);
        c[3] = fmaf(c[3], om, b1);
      }
      if (res) {  // uniform
#pragma unroll
        for (int q = 0; q < 4; ++q) x[j][q] += act_fast(act, c[q]);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) x[j][q] = act_fast(act, c[q]);
      }
    }
  }
}

// rows [16][ld] FP32 <-> C-fragment registers.
template <int H>
__device__ __forceinline__ void tile_load(float (&x)[H / 8][4], const float* rows, int ld, int nrows) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j < H / 8; ++j) {
    const int c = 8 * j + 2 * t;
    x[j][0] = g < nrows ? rows[g * ld + c] : 0.f;
    x[j][1] = g < nrows ? rows[g * ld + c + 1] : 0.f;
    x[j][2] = g + 8 < nrows ? rows[(g + 8) * ld + c] : 0.f;
    x[j][3] = g + 8 < nrows ? rows[(g + 8) * ld + c + 1] : 0.f;
  }
}

template <int H>
__device__ __forceinline__ void tile_store(const float (&x)[H / 8][4], float* rows, int ld, int nrows) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j < H / 8; ++j) {
    const int c = 8 * j + 2 * t;
    if (g < nrows) {
      rows[g * ld + c] = x[j][0];
      rows[g * ld + c + 1] = x[j][1];
    }
    if (g + 8 < nrows) {
      rows[(g + 8) * ld + c] = x[j][2];
      rows[(g + 8) * ld + c + 1] = x[j][3];
    }
  }
}

}  // namespace scale
