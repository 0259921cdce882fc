// ace.cu -- the ACE network (Sec. II "ACE", Eq. ACE) for batches of configurations:
//   H0_i     = E_i[n_i]
//   H(l+1)   = LN( H(l) + SiLU(Conv_l(H(l))) )            l < n_conv (3x3, the Hamiltonian's
//                                                          boundary conditions)
//   H(l+1)   = act( H(l) W_l + b_l )                       site-wise layers (Eq. MLP), width h_mlp
//   Phi[a][k] = M0[o_a][k] + proj_b[s*Ne+k] + H(L)_i . proj_w[:, s*Ne+k]   (o_a = s*N + i
//                                                          ascending; FP64 for the LU)
// LN normalises each site's channel vector: mean and biased variance over the channels,
// (u - mean) / sqrt(var + eps) * gamma + beta.
//
// A change at one site moves the features of every site after enough blocks, so every
// configuration -- each n' of a local energy included -- is a fresh forward (the O(N^4)
// route of Sec. III.A). The forward is dense work: a conv block is a GEMM of
// (configurations x sites) rows against 9 stacked h x h weights with the rows gathered
// by neighbour offset.
//
// Implementations of a layer:
//   k_ace_conv_tc (mixed mode: the ACE conv blocks of width 48, 144 or 192, the wide SCALE
//               conv of width 384 or 640, and the site-wise layers that follow them while
//               their output widths are multiples of 128): the 5th-generation tensor cores.
//               One CTA of 256 threads (two per row) owns 128 rows (TMEM lanes) and a tile
//               of N output channels (TMEM columns; the whole width for a normalised block,
//               else 128 to 192); the column tiles of the same rows are adjacent in the
//               grid, so they share the gathered rows through L2. The K loop runs over (offset d, 8-channel chunk) stages
//               in a 6-slot shared-memory ring with 4 stages of copies in flight: each
//               thread gathers its row's 8 input channels, hi or lo part, from the
//               neighbour site with 16-byte cp.async (zero fill past an open edge),
//               the pre-split weight tile arrives by one bulk copy per half (hi, lo) on an
//               mbarrier, and one thread issues the three TF32 products
//               x_hi W_hi + x_lo W_hi + x_hi W_lo per K=8 step (tcgen05.mma, FP32
//               accumulation in TMEM) and commits them to the stage's mbarrier. Between two
//               tensor-core layers the activations are stored already split (hi, lo).
//               Epilogue per thread = half a row, held in registers: the residual (loaded
//               while the last MMAs finish), tcgen05.ld of the accumulator in 8-column
//               chunks, bias, activation, the layer normalisation (mean, then the centred
//               variance, the two halves combined through shared memory), the split for
//               the next layer.
//   k_ace_mma   (mixed mode, the other site-wise layers): mma.sync tensor cores, every
//               product as three TF32 products of a hi/lo split (x_hi W_hi + x_lo W_hi + x_hi W_lo, FP32
//               accumulation, about 2^-21 relative per layer). A warp owns 16 rows and
//               WC warps share a row group's output columns; the A operand is gathered from
//               the neighbour sites' rows (L1/L2), the weights come as pre-split fragments.
//               Bias, residual, activation and the layer normalisation run in the epilogue
//               on the accumulators (a row's channels live in one lane quad when WC = 1).
//   k_ace_layer (FP64 mode, and other widths in FP32): one warp per row, CUDA cores, the
//               same sum order as the definition (bias, then offsets, then channels).
#include <algorithm>

#include "mlp_mma.cuh"
#include "scale_internal.cuh"
#include "tcgen05.cuh"

namespace scale {

namespace {

constexpr int kAceRowsGeneric = 8;  // rows (one warp each) per CTA of k_ace_layer

template <typename T>
struct AceNet {
  int h, L, n_conv, act, per_site, stencil;
  double eps;
  int cin[kMaxLayers], cout[kMaxLayers], ks[kMaxLayers];
  const T* embed;
  const T* kernel[kMaxLayers];
  const T* bias[kMaxLayers];
  const T* ln_g[kMaxLayers];  // nullptr for the site-wise layers
  const T* ln_b[kMaxLayers];
  const T* proj_w;            // [c_last][2 Ne]
  const T* proj_b;            // [2 Ne]
  const T* M0;                // [2N][Ne]
};

// Flat layout: embed; per layer kernel [k][k][c_in][c_out], bias [c_out], and for the conv
// blocks ln gamma [c_out], ln beta [c_out]; proj_w [c_last][2Ne]; proj_b [2Ne].
template <typename T>
AceNet<T> make_ace_net(const scale_ctx* c) {
  AceNet<T> n{};
  const scale_arch& a = c->arch;
  n.h = c->h;
  n.L = c->L;
  n.n_conv = a.n_conv;
  n.act = a.act;
  n.per_site = a.per_site_embed;
  n.stencil = a.stencil;
  n.eps = a.ln_eps;
  const bool ln = a.family == SCALE_FAMILY_ACE;
  const T* base = c->fp64 ? (const T*)c->params64 : (const T*)c->params32;
  int64_t p = 0;
  n.embed = base;
  p += (int64_t)(a.per_site_embed ? c->N : 1) * 4 * c->h;
  for (int l = 0; l < c->L; ++l) {
    n.ks[l] = a.ksize[l];
    n.cin[l] = ace_width_in(a, l);
    n.cout[l] = ace_width_out(a, l);
    n.kernel[l] = base + p;
    p += (int64_t)stencil_taps(a.stencil, n.ks[l]) * n.cin[l] * n.cout[l];
    n.bias[l] = base + p;
    p += n.cout[l];
    n.ln_g[l] = n.ln_b[l] = nullptr;
    if (ln && l < a.n_conv) {
      n.ln_g[l] = base + p;
      p += n.cout[l];
      n.ln_b[l] = base + p;
      p += n.cout[l];
    }
  }
  n.proj_w = base + p;
  p += (int64_t)n.cout[c->L - 1] * 2 * c->Ne;
  n.proj_b = base + p;
  n.M0 = c->fp64 ? (const T*)c->M0_64 : (const T*)c->M0_32;
  return n;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// H0 rows [C][N][h] from the embedding tables.
template <typename T>
__global__ void k_ace_embed(int N, int h, int per_site, const T* __restrict__ embed, const int8_t* __restrict__ occ,
                            long long total, T* __restrict__ out, const int* __restrict__ vcfg) {
  if (vcfg) total = min(total, (long long)*vcfg * N * h);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const long long row = q / h;
    const int c = (int)(q - row * h);
    const int i = (int)(row % N);
    const int s = occ[row] & 3;
    out[q] = embed[((size_t)(per_site ? i : 0) * 4 + s) * h + c];
  }
}

// One layer on CUDA cores, one warp per row (configuration, site); 16 output channels per
// lane at a time (chunks of 512; a normalised layer has at most 512). The taps run over the
// k x k box in row-major order, skipping the offsets outside the stencil.
template <typename T>
__global__ void __launch_bounds__(32 * kAceRowsGeneric) k_ace_layer(
    Lattice lat, const T* __restrict__ K, const T* __restrict__ bias, const T* __restrict__ gam,
    const T* __restrict__ bet, int ks, int stencil, int cin, int cout, int res, int act, double eps,
    const T* __restrict__ in, T* __restrict__ out, long long rows, const int* __restrict__ vcfg) {
  constexpr int MQ = kAceMaxHMlp / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (vcfg) rows = min(rows, (long long)*vcfg * lat.N);
  const long long R = (long long)blockIdx.x * kAceRowsGeneric + warp;
  if (R >= rows) return;  // whole warp
  const int N = lat.N;
  const long long cfg = R / N;
  const int i = (int)(R - cfg * N);
  const int r = (ks - 1) / 2;
  const T* self = in + (size_t)R * cin;
  T* o = out + (size_t)R * cout;
  for (int cb = 0; cb < cout; cb += 32 * MQ) {
    T acc[MQ];
#pragma unroll
    for (int q = 0; q < MQ; ++q) {
      const int co = cb + lane + 32 * q;
      acc[q] = co < cout ? bias[co] : T(0);
    }
    int tap = 0;
    for (int d = 0; d < ks * ks; ++d) {
      const int dx = d % ks - r, dy = d / ks - r;
      if (!stencil_has(stencil, ks, dx, dy)) continue;
      const int t = tap++;
      const int j = site_off(lat, i, dx, dy);
      if (j < 0) continue;  // zero padding past an open edge
      const T* x = in + ((size_t)cfg * N + j) * cin;
      const T* w = K + (size_t)t * cin * cout;
      for (int ci = 0; ci < cin; ++ci) {
        const T xv = x[ci];
        const T* wr = w + (size_t)ci * cout;
#pragma unroll
        for (int q = 0; q < MQ; ++q) {
          const int co = cb + lane + 32 * q;
          if (co < cout) acc[q] += xv * wr[co];
        }
      }
    }
    T s = T(0);
#pragma unroll
    for (int q = 0; q < MQ; ++q) {
      const int co = cb + lane + 32 * q;
      if (co < cout) {
        acc[q] = (res ? self[co] : T(0)) + act_fn<T>(act, acc[q]);
        s += acc[q];
      }
    }
    if (gam) {  // layer normalisation over this site's channels (cout <= 512: one chunk)
      const T mean = warp_sum(s) / T(cout);
      T v = T(0);
#pragma unroll
      for (int q = 0; q < MQ; ++q) {
        const int co = cb + lane + 32 * q;
        if (co < cout) v += (acc[q] - mean) * (acc[q] - mean);
      }
      v = warp_sum(v) / T(cout);
      const T inv = T(1) / sqrt(v + T(eps));
#pragma unroll
      for (int q = 0; q < MQ; ++q) {
        const int co = cb + lane + 32 * q;
        if (co < cout) acc[q] = (acc[q] - mean) * inv * gam[co] + bet[co];
      }
    }
#pragma unroll
    for (int q = 0; q < MQ; ++q) {
      const int co = cb + lane + 32 * q;
      if (co < cout) o[co] = acc[q];
    }
  }
}

// Pre-split weight fragments of one layer, [tap][kk][nt][lane] {b0_hi, b1_hi, b0_lo, b1_lo},
// with the k index of each 8-wide step permuted (logical t -> channel 2t, logical t+4 ->
// channel 2t+1) so that a lane's two A entries are adjacent channels (one 8-byte load).
__global__ void k_ace_build_frag(const float* __restrict__ K, int taps, int cin, int cout, WFrag* __restrict__ out) {
  const int KT = cin / 8, NT = cout / 8;
  const size_t total = (size_t)taps * KT * NT * 32;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int lane = (int)(q % 32);
    size_t r = q / 32;
    const int nt = (int)(r % NT);
    r /= NT;
    const int kk = (int)(r % KT);
    const int d = (int)(r / KT);
    const int g = lane >> 2, t = lane & 3;
    const float* w = K + (size_t)d * cin * cout;
    const float b0 = w[(size_t)(8 * kk + 2 * t) * cout + 8 * nt + g];
    const float b1 = w[(size_t)(8 * kk + 2 * t + 1) * cout + 8 * nt + g];
    WFrag f;
    split_tf32(b0, f.v[0], f.v[2]);
    split_tf32(b1, f.v[1], f.v[3]);
    out[q] = f;
  }
}

// One layer on the tensor cores. CTA: 8 warps = (8 / WC) row groups of 16 rows x WC column
// groups of NTW n-tiles; cout = 8 NTW WC. LN (WC = 1 only): layer normalisation of each row
// in the epilogue (the row's channels are spread over the 4 lanes of a quad).
template <int NTW, int WC, bool LN>
__global__ void __launch_bounds__(256, (NTW > 18 || NTW == 16 ? 1 : 2)) k_ace_mma(
    Lattice lat, const WFrag* __restrict__ frag, const float* __restrict__ bias, const float* __restrict__ gam,
    const float* __restrict__ bet, int ks, int stencil, int cin, int res, int act, float eps,
    const float* __restrict__ in, float* __restrict__ out, long long rows, const int* __restrict__ vcfg) {
  static_assert(!LN || WC == 1, "the epilogue normalisation needs a row's channels in one warp");
  constexpr int NT = NTW * WC, COUT = 8 * NT, WR = 8 / WC, ROWS = 16 * WR;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int wr = warp / WC, wc = warp % WC;
  const int N = lat.N;
  if (vcfg) rows = min(rows, (long long)*vcfg * N);
  const long long r0 = (long long)blockIdx.x * ROWS + wr * 16 + g, r1 = r0 + 8;
  const bool v0 = r0 < rows, v1 = r1 < rows;
  const long long c0 = v0 ? r0 / N : 0, c1 = v1 ? r1 / N : 0;
  const int i0 = v0 ? (int)(r0 - c0 * N) : 0, i1 = v1 ? (int)(r1 - c1 * N) : 0;
  const int col0 = 8 * wc * NTW + 2 * t;

  float acc[NTW][4];
#pragma unroll
  for (int j = 0; j < NTW; ++j) {
    const float b0 = bias[col0 + 8 * j], b1 = bias[col0 + 8 * j + 1];
    acc[j][0] = b0;
    acc[j][1] = b1;
    acc[j][2] = b0;
    acc[j][3] = b1;
  }
  const int KT = cin / 8, rad = (ks - 1) / 2;
  int tap = 0;
  for (int d = 0; d < ks * ks; ++d) {
    const int dx = d % ks - rad, dy = d / ks - rad;
    if (!stencil_has(stencil, ks, dx, dy)) continue;
    const int tp = tap++;
    const int j0 = v0 ? site_off(lat, i0, dx, dy) : -1;
    const int j1 = v1 ? site_off(lat, i1, dx, dy) : -1;
    const float* p0 = j0 >= 0 ? in + ((size_t)c0 * N + j0) * cin + 2 * t : nullptr;
    const float* p1 = j1 >= 0 ? in + ((size_t)c1 * N + j1) * cin + 2 * t : nullptr;
    const WFrag* fd = frag + (size_t)tp * KT * NT * 32 + (size_t)wc * NTW * 32 + lane;
    for (int kk = 0; kk < KT; ++kk) {
      const float2 x0 = p0 ? __ldg(reinterpret_cast<const float2*>(p0 + 8 * kk)) : make_float2(0.f, 0.f);
      const float2 x1 = p1 ? __ldg(reinterpret_cast<const float2*>(p1 + 8 * kk)) : make_float2(0.f, 0.f);
      uint32_t ah[4], al[4];
      split_tf32(x0.x, ah[0], al[0]);  // (g,   logical t)   = channel 8kk + 2t
      split_tf32(x1.x, ah[1], al[1]);  // (g+8, logical t)
      split_tf32(x0.y, ah[2], al[2]);  // (g,   logical t+4) = channel 8kk + 2t + 1
      split_tf32(x1.y, ah[3], al[3]);  // (g+8, logical t+4)
      const WFrag* fk = fd + (size_t)kk * NT * 32;
#pragma unroll
      for (int j = 0; j < NTW; ++j) {
        const WFrag w = fk[j * 32];
        mma_tf32(acc[j], ah, w.v[0], w.v[1]);
        mma_tf32(acc[j], al, w.v[0], w.v[1]);
        mma_tf32(acc[j], ah, w.v[2], w.v[3]);
      }
    }
  }
  // epilogue: residual + activation, then the normalisation of each row
  float s0 = 0.f, s1 = 0.f;
#pragma unroll
  for (int j = 0; j < NTW; ++j) {
    const int col = col0 + 8 * j;
    float2 x0 = make_float2(0.f, 0.f), x1 = make_float2(0.f, 0.f);
    if (res) {
      if (v0) x0 = *reinterpret_cast<const float2*>(in + (size_t)r0 * cin + col);
      if (v1) x1 = *reinterpret_cast<const float2*>(in + (size_t)r1 * cin + col);
    }
    acc[j][0] = x0.x + act_fast(act, acc[j][0]);
    acc[j][1] = x0.y + act_fast(act, acc[j][1]);
    acc[j][2] = x1.x + act_fast(act, acc[j][2]);
    acc[j][3] = x1.y + act_fast(act, acc[j][3]);
    s0 += acc[j][0] + acc[j][1];
    s1 += acc[j][2] + acc[j][3];
  }
  if constexpr (LN) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
    s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
    const float m0 = s0 * (1.f / COUT), m1 = s1 * (1.f / COUT);
    float q0 = 0.f, q1 = 0.f;
#pragma unroll
    for (int j = 0; j < NTW; ++j) {
      q0 += (acc[j][0] - m0) * (acc[j][0] - m0) + (acc[j][1] - m0) * (acc[j][1] - m0);
      q1 += (acc[j][2] - m1) * (acc[j][2] - m1) + (acc[j][3] - m1) * (acc[j][3] - m1);
    }
    q0 += __shfl_xor_sync(0xffffffffu, q0, 1);
    q0 += __shfl_xor_sync(0xffffffffu, q0, 2);
    q1 += __shfl_xor_sync(0xffffffffu, q1, 1);
    q1 += __shfl_xor_sync(0xffffffffu, q1, 2);
    const float inv0 = 1.f / sqrtf(q0 * (1.f / COUT) + eps), inv1 = 1.f / sqrtf(q1 * (1.f / COUT) + eps);
#pragma unroll
    for (int j = 0; j < NTW; ++j) {
      const int col = col0 + 8 * j;
      const float ga = gam[col], gb = gam[col + 1], ba = bet[col], bb = bet[col + 1];
      acc[j][0] = (acc[j][0] - m0) * inv0 * ga + ba;
      acc[j][1] = (acc[j][1] - m0) * inv0 * gb + bb;
      acc[j][2] = (acc[j][2] - m1) * inv1 * ga + ba;
      acc[j][3] = (acc[j][3] - m1) * inv1 * gb + bb;
    }
  }
#pragma unroll
  for (int j = 0; j < NTW; ++j) {
    const int col = col0 + 8 * j;
    if (v0) *reinterpret_cast<float2*>(out + (size_t)r0 * COUT + col) = make_float2(acc[j][0], acc[j][1]);
    if (v1) *reinterpret_cast<float2*>(out + (size_t)r1 * COUT + col) = make_float2(acc[j][2], acc[j][3]);
  }
}

// ---- conv blocks on tcgen05 ---------------------------------------------------------------
constexpr int kTcRows = 128;  // M of a tile = TMEM lanes
constexpr int kTcThreads = 256;  // two threads per row
constexpr int kTcKC = 8;      // input channels per pipeline stage (one K = 8 MMA step)
constexpr int kTcStages = 6;  // shared-memory ring
constexpr int kTcAhead = 4;   // stages whose copies are in flight ahead of the MMA
constexpr uint32_t kTcWaitPolls = 1u << 24;  // bound of every mbarrier wait

// Byte offset of element (r, k) of an [R x 8] tf32 tile in the K-major core-matrix layout:
// core matrix (r / 8, k / 4) at ((r / 8) * 2 + k / 4) * 128, its row r % 8 at 16 bytes.
// Neighbours along K are 128 bytes apart (descriptor LBO), along rows 256 (SBO).
__host__ __device__ constexpr uint32_t tc_off(int r, int k) {
  return (uint32_t)(((r >> 3) * 2 + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4);
}
constexpr uint32_t kTcLBO = 128, kTcSBO = 256;

// Activation of the tensor-core conv epilogue: SiLU as z / (1 + e^-z) with the fast
// reciprocal-based division (the exponent capped so the denominator stays finite).
__device__ __forceinline__ float act_tc(int act, float z) {
  if (act == SCALE_ACT_SILU) return __fdividef(z, 1.f + __expf(fminf(-z, 80.f)));
  return tanh_f32(z);
}

template <int N>
struct TcShape {
  static constexpr uint32_t A_BYTES = kTcRows * kTcKC * 4;  // one half (hi or lo) of the A tile
  static constexpr uint32_t B_BYTES = N * kTcKC * 4;        // one half of the weight tile
  static constexpr uint32_t STAGE = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr uint32_t SMEM = kTcStages * STAGE + 2 * kTcStages * 8 + 16 + 1024;  // + barriers, slot, alignment
  static constexpr uint32_t TCOLS = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
};

// Weight tiles of a conv layer in the shared-memory image the MMA reads:
// [tap d][chunk kc][hi, lo][N rows (output channel) x 8 (input channel)] core-matrix layout;
// the rows [c0, c0 + n) of a tile are the contiguous bytes [32 c0, 32 (c0 + n)).
__global__ void k_ace_build_bimg(const float* __restrict__ K, int CI, int N, int taps, float* __restrict__ out) {
  const int KC = CI / kTcKC;
  const size_t total = (size_t)taps * KC * 2 * N * kTcKC;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(q % kTcKC);
    size_t r = q / kTcKC;
    const int n = (int)(r % N);
    r /= N;
    const int part = (int)(r % 2);
    r /= 2;
    const int kc = (int)(r % KC);
    const int d = (int)(r / KC);
    const float w = K[((size_t)d * CI + kc * kTcKC + k) * N + n];
    uint32_t hi, lo;
    split_tf32(w, hi, lo);
    const size_t tile = (((size_t)d * KC + kc) * 2 + part) * N * kTcKC;
    out[tile + tc_off(n, k) / 4] = __uint_as_float(part ? lo : hi);
  }
}

// H0 rows split for the tensor cores: out_hi = tf32(E), out_lo = tf32(E - out_hi).
__global__ void k_ace_embed_split(int N, int h, int per_site, const float* __restrict__ embed,
                                  const int8_t* __restrict__ occ, long long total, float* __restrict__ out_hi,
                                  float* __restrict__ out_lo, const int* __restrict__ vcfg) {
  if (vcfg) total = min(total, (long long)*vcfg * N * h);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const long long row = q / h;
    const int c = (int)(q - row * h);
    const int i = (int)(row % N);
    const float e = embed[((size_t)(per_site ? i : 0) * 4 + (occ[row] & 3)) * h + c];
    uint32_t hi, lo;
    split_tf32(e, hi, lo);
    out_hi[q] = __uint_as_float(hi);
    out_lo[q] = __uint_as_float(lo);
  }
}

// One conv layer (ks x ks stencil, C -> C channels) on tcgen05: ACE blocks with the layer
// normalisation in the epilogue (LN, one column tile of N = C), or the wide SCALE conv (no
// normalisation, column tiles of N: blockIdx.y selects columns [N y, N y + N)). out_lo ==
// nullptr writes plain FP32 rows to out_hi (the input of the site-wise layers). err: set when
// a wait ran out. 256 threads: thread t serves row t % 128 -- copies of its hi (t < 128) or
// lo half, and in the epilogue the tile's columns [0, N/2) (warps 0-3) or [N/2, N) (warps
// 4-7); a warp reads the TMEM lanes of its quarter (warp % 4).
template <int N, bool LN>
__global__ void __launch_bounds__(kTcThreads, (N > 144 ? 1 : 2)) k_ace_conv_tc(
    Lattice lat, const float* __restrict__ bimg, const float* __restrict__ bias, const float* __restrict__ gam,
    const float* __restrict__ bet, int act, float eps, int C, int CO, int res, int ks, int stencil, int taps,
    const float* __restrict__ in_hi, const float* __restrict__ in_lo, float* __restrict__ out_hi,
    float* __restrict__ out_lo, long long row0, long long rows, int* __restrict__ err,
    const int* __restrict__ vcfg) {
  // C input channels (K = taps x C), CO output channels (this CTA: [cb, cb + N)); res: add the
  // input row (C == CO). A normalised block is one tile wide: C == CO == N.
  if constexpr (LN) C = CO = N;
  using S = TcShape<N>;
  const int KC = C / kTcKC;
  const int STEPS = taps * KC;
  // Grid (column tile, row tile): the CO / N column tiles of the same 128 rows are adjacent
  // in launch order and run side by side, so all but the first read the rows from L2.
  const int cb = blockIdx.x * N;  // first output column of this CTA
  constexpr int H2 = N / 2;  // epilogue columns per thread
  constexpr uint32_t IDESC = tc::idesc_tf32<kTcRows, N>();
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte aligned ring (descriptors address 16-byte units; core matrices 128 bytes)
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kTcStages * S::STAGE);
  uint64_t* done = full + kTcStages;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + kTcStages);
  __shared__ int s_abort;
  __shared__ float s_sum[2][kTcRows], s_sq[2][kTcRows];  // per-half row sums for the normalisation
  const int tid = threadIdx.x, warp = tid >> 5, row = tid & (kTcRows - 1), part = tid >> 7;
  const int Ns = lat.N;
  // rows past the valid configurations of a chunk (vcfg: their count on the device): a tile
  // that holds none of them leaves before any barrier, mbarrier or TMEM allocation
  if (vcfg) rows = min(rows, (long long)*vcfg * Ns);
  if (row0 + (long long)blockIdx.y * kTcRows >= rows) return;
  const long long R = row0 + (long long)blockIdx.y * kTcRows + row;
  const bool valid = R < rows;
  const long long cfg = valid ? R / Ns : 0;
  const int site = valid ? (int)(R - cfg * Ns) : 0;

  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&done[s], 1);
    }
    tc::mbar_fence_init();
    s_abort = 0;
  }
  if (warp == 0) tc::tmem_alloc(tslot, S::TCOLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;

  // Copies of the stages in order, one per call; each call closes one cp.async group
  // (empty past the last stage). The neighbour row of the current tap is recomputed only
  // when the tap changes (every KC stages).
  const float* in_part = part ? in_lo : in_hi;
  int is = 0, id = 0, ikc = 0;
  size_t isrc = 0;
  uint32_t inb = 0;
  auto tap_row = [&](int d) {
    int dx, dy;
    stencil_tap(stencil, ks, d, dx, dy);
    const int j = valid ? site_off(lat, site, dx, dy) : -1;
    isrc = j >= 0 ? ((size_t)cfg * Ns + j) * C : 0;
    inb = j >= 0 ? 16u : 0u;  // zero fill past an open edge or the last row
  };
  tap_row(0);
  const uint32_t a_off0 = part * S::A_BYTES + tc_off(row, 0), a_off1 = part * S::A_BYTES + tc_off(row, 4);
  auto issue_next = [&]() {
    if (is < STEPS) {
      const int b = is % kTcStages;
      unsigned char* st = smem + b * S::STAGE;
      const size_t src = isrc + (size_t)ikc * kTcKC;
      tc::cp_async16_zfill(st + a_off0, in_part + src, inb);
      tc::cp_async16_zfill(st + a_off1, in_part + src + 4, inb);
      if (tid == 0) {
        const float* w = bimg + ((size_t)id * KC + ikc) * 2 * CO * kTcKC + (size_t)cb * kTcKC;
        tc::mbar_arrive_expect_tx(&full[b], 2 * S::B_BYTES);
        tc::bulk_g2s(st + 2 * S::A_BYTES, w, S::B_BYTES, &full[b]);
        tc::bulk_g2s(st + 2 * S::A_BYTES + S::B_BYTES, w + CO * kTcKC, S::B_BYTES, &full[b]);
      }
      ++is;
      if (++ikc == KC) {
        ikc = 0;
        if (++id < taps) tap_row(id);
      }
    }
    tc::cp_async_commit();
  };

#pragma unroll 1
  for (int p = 0; p < kTcAhead; ++p) issue_next();
#pragma unroll 1
  for (int s = 0; s < STEPS; ++s) {
    const int b = s % kTcStages;
    const int s1 = s + kTcAhead;
    // the ring slot of stage s1 last held stage s1 - kTcStages (two MMA stages back)
    bool ok = true;
    if (s1 < STEPS && s1 >= kTcStages)
      ok = tc::mbar_wait(&done[s1 % kTcStages], (uint32_t)((s1 / kTcStages) - 1) & 1u, kTcWaitPolls);
    if (ok) {
      issue_next();  // stage s1
    } else {
      s_abort = 1;
      tc::cp_async_commit();
    }
    tc::cp_async_wait<kTcAhead>();  // this thread's copies of stage s have landed
    tc::fence_proxy_async();        // ... and are visible to the tensor core
    __syncthreads();
    if (s_abort) break;
    if (tid == 0) {
      if (!tc::mbar_wait(&full[b], (uint32_t)(s / kTcStages) & 1u, kTcWaitPolls)) {
        s_abort = 1;
      } else {
        tc::fence_after_sync();
        const uint32_t a0 = tc::smem_u32(smem + b * S::STAGE);
        const uint64_t ah = tc::smem_desc_kmajor(a0, kTcLBO, kTcSBO);
        const uint64_t al = tc::smem_desc_kmajor(a0 + S::A_BYTES, kTcLBO, kTcSBO);
        const uint64_t bh = tc::smem_desc_kmajor(a0 + 2 * S::A_BYTES, kTcLBO, kTcSBO);
        const uint64_t bl = tc::smem_desc_kmajor(a0 + 2 * S::A_BYTES + S::B_BYTES, kTcLBO, kTcSBO);
        tc::mma_tf32(tmem, ah, bh, IDESC, s > 0 ? 1u : 0u);
        tc::mma_tf32(tmem, al, bh, IDESC, 1u);
        tc::mma_tf32(tmem, ah, bl, IDESC, 1u);
        tc::mma_commit(&done[b]);
      }
    }
  }
  // this thread's half of the tile's residual row (independent of the MMAs: loaded under them);
  // the 256-column tiles (site-wise layers, no residual) stream their epilogue instead
  constexpr bool kStream = N == 256;
  const int c0 = part * H2;
  float u[kStream ? 1 : H2];
  if constexpr (kStream) {
    u[0] = 0.f;
  } else if (LN || res) {  // the normalised conv blocks are residual
    const float* xh = in_hi + (size_t)(valid ? R : 0) * C + cb + c0;
    const float* xl = in_lo + (size_t)(valid ? R : 0) * C + cb + c0;
#pragma unroll
    for (int c = 0; c < H2; c += 4) {
      const float4 h4 = __ldg(reinterpret_cast<const float4*>(xh + c));
      const float4 l4 = __ldg(reinterpret_cast<const float4*>(xl + c));
      u[c] = h4.x + l4.x;
      u[c + 1] = h4.y + l4.y;
      u[c + 2] = h4.z + l4.z;
      u[c + 3] = h4.w + l4.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < H2; ++c) u[c] = 0.f;
  }
  (void)u;
  if (!s_abort && tid == 0) {
    const int sl = STEPS - 1;
    if (!tc::mbar_wait(&done[sl % kTcStages], (uint32_t)(sl / kTcStages) & 1u, kTcWaitPolls)) s_abort = 1;
  }
  tc::cp_async_wait<0>();
  __syncthreads();
  tc::fence_after_sync();
  const bool run = !s_abort;
  if constexpr (kStream) {  // 8 columns at a time: TMEM -> bias, activation -> (split) store
    if (run) {
      const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16) + c0;
#pragma unroll 1
      for (int cc = 0; cc < H2 / 8; ++cc) {
        float z[8];
        tc::tmem_ld8(trow + cc * 8, z);
#pragma unroll
        for (int q = 0; q < 8; ++q) z[q] = act_tc(act, z[q] + __ldg(bias + cb + c0 + cc * 8 + q));
        if (valid) {
          const size_t o = (size_t)R * CO + cb + c0 + cc * 8;
          if (out_lo) {
            uint32_t hi[8], lo[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) split_tf32(z[e], hi[e], lo[e]);
#pragma unroll
            for (int e = 0; e < 8; e += 4) {
              *reinterpret_cast<float4*>(out_hi + o + e) = make_float4(
                  __uint_as_float(hi[e]), __uint_as_float(hi[e + 1]), __uint_as_float(hi[e + 2]), __uint_as_float(hi[e + 3]));
              *reinterpret_cast<float4*>(out_lo + o + e) = make_float4(
                  __uint_as_float(lo[e]), __uint_as_float(lo[e + 1]), __uint_as_float(lo[e + 2]), __uint_as_float(lo[e + 3]));
            }
          } else {
#pragma unroll
            for (int e = 0; e < 8; e += 4)
              *reinterpret_cast<float4*>(out_hi + o + e) = make_float4(z[e], z[e + 1], z[e + 2], z[e + 3]);
          }
        }
      }
    } else if (tid == 0) {
      atomicExch(err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, S::TCOLS);
    return;
  }
  if (run) {
    const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16) + c0;
#pragma unroll
    for (int cc = 0; cc < H2 / 8; ++cc) {
      float z[8];
      tc::tmem_ld8(trow + cc * 8, z);
#pragma unroll
      for (int q = 0; q < 8; ++q) u[cc * 8 + q] += act_tc(act, z[q] + __ldg(bias + cb + c0 + cc * 8 + q));
    }
    if constexpr (LN) {
      float s1 = 0.f;
#pragma unroll
      for (int c = 0; c < H2; ++c) s1 += u[c];
      s_sum[part][row] = s1;
    }
  }
  float mean = 0.f, inv = 1.f;
  if constexpr (LN) {
    __syncthreads();
    if (run) {
      mean = (s_sum[0][row] + s_sum[1][row]) * (1.f / N);
      float s2 = 0.f;
#pragma unroll
      for (int c = 0; c < H2; ++c) s2 += (u[c] - mean) * (u[c] - mean);
      s_sq[part][row] = s2;
    }
    __syncthreads();
    if (run) inv = 1.f / sqrtf((s_sq[0][row] + s_sq[1][row]) * (1.f / N) + eps);
  }
  if (run) {
#pragma unroll
    for (int c = 0; c < H2; c += 4) {
      float y[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if constexpr (LN) y[e] = (u[c + e] - mean) * inv * __ldg(gam + c0 + c + e) + __ldg(bet + c0 + c + e);
        else y[e] = u[c + e];
      }
      if (valid) {
        const size_t o = (size_t)R * CO + cb + c0 + c;
        if (out_lo) {
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) split_tf32(y[e], hi[e], lo[e]);
          *reinterpret_cast<float4*>(out_hi + o) = make_float4(__uint_as_float(hi[0]), __uint_as_float(hi[1]),
                                                               __uint_as_float(hi[2]), __uint_as_float(hi[3]));
          *reinterpret_cast<float4*>(out_lo + o) = make_float4(__uint_as_float(lo[0]), __uint_as_float(lo[1]),
                                                               __uint_as_float(lo[2]), __uint_as_float(lo[3]));
        } else {
          *reinterpret_cast<float4*>(out_hi + o) = make_float4(y[0], y[1], y[2], y[3]);
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, S::TCOLS);
}

template <int N, bool LN>
cudaError_t run_conv_tc(cudaStream_t st, const Lattice& lat, const float* bimg, const float* bias, const float* g,
                        const float* be, int act, float eps, int C, int CO, int res, int ks, int stencil,
                        const float* in_hi, const float* in_lo, float* out_hi, float* out_lo, long long rows,
                        int* err, const int* vcfg) {
  using S = TcShape<N>;
  cudaError_t e =
      cudaFuncSetAttribute(k_ace_conv_tc<N, LN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
  if (e != cudaSuccess) return e;
  // rows [row0, rows) per launch, at most 65535 row tiles (the grid's y limit) each
  const long long tiles = (rows + kTcRows - 1) / kTcRows;
  for (long long t0 = 0; t0 < tiles; t0 += 65535) {
    const dim3 grid((unsigned)(CO / N), (unsigned)std::min<long long>(65535, tiles - t0));
    k_ace_conv_tc<N, LN><<<grid, kTcThreads, S::SMEM, st>>>(lat, bimg, bias, g, be, act, eps, C, CO, res, ks,
                                                            stencil, stencil_taps(stencil, ks), in_hi, in_lo,
                                                            out_hi, out_lo, t0 * kTcRows, rows, err, vcfg);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Conv layers on tcgen05: ACE blocks of width 48, 144 or 192 (3x3 box, one column tile,
// normalisation in the epilogue); the wide SCALE conv of width 384 (two tiles of 192) or 640
// (four tiles of 160), 3x3 box or the 5x5 plus.
bool tc_width(int h) { return h == 48 || h == 144 || h == 192; }
bool tc_wide_width(int h) { return h == 384 || h == 640; }
// Site-wise layers on tcgen05 (1x1, no residual): input width a multiple of 8, output width a
// multiple of 128 (tiles of 128 columns, two CTAs per SM).
bool tc_sitewise(int cin, int cout) { return cin % kTcKC == 0 && cout % 128 == 0; }

cudaError_t launch_conv_tc(const scale_ctx* c, const Lattice& lat, bool ln, int cin, int cout, int res, int ks,
                           const float* bimg, const float* bias, const float* g, const float* be, int act, float eps,
                           const float* in_hi, const float* in_lo, float* out_hi, float* out_lo, long long rows,
                           const int* vcfg) {
  const int st = c->arch.stencil;
#define SCALE_TC(NT, LNV) \
  run_conv_tc<NT, LNV>(c->stream, lat, bimg, bias, g, be, act, eps, cin, cout, res, ks, st, in_hi, in_lo, \
                       out_hi, out_lo, rows, c->ace_err, vcfg)
  if (ln) {
    if (cout == 48) return SCALE_TC(48, true);
    if (cout == 144) return SCALE_TC(144, true);
    return SCALE_TC(192, true);
  }
  if (ks > 1 && cout == 384) return SCALE_TC(192, false);
  if (ks > 1 && cout == 640) return SCALE_TC(160, false);
  // site-wise layers without residual: 256-column tiles where the width allows (twice the
  // MMA work per pipeline stage, the rows read half as often); else 128
  if (ks == 1 && !res && cout % 256 == 0) return SCALE_TC(256, false);
  return SCALE_TC(128, false);
#undef SCALE_TC
}

// Slater matrix rows of the occupied orbitals in ascending order (FP64 output):
//   Phi[a][k] = M0[o_a][k] + proj_b[s Ne + k] + sum_c H(L)_i[c] proj_w[c][s Ne + k].
// A register-tiled GEMM per configuration: CTA (row tile, column tile, configuration) of
// 64 x 64 outputs, rows of one spin only (the up rows precede the down rows in ascending
// order), 4 x 4 outputs per thread, channels staged 32 at a time through shared memory.
// A configuration with another electron count gets a zero matrix (singular); after a
// tensor-core layer gave up waiting, NaN.
constexpr int kPhiT = 64, kPhiK = 32;

template <typename T>
__global__ void __launch_bounds__(256) k_ace_phi(Lattice lat, AceNet<T> net, int hl, const int8_t* __restrict__ occ,
                                                 const T* __restrict__ HL, const int* __restrict__ err,
                                                 double* __restrict__ phi, const int* __restrict__ vcfg) {
  extern __shared__ int olist[];  // [2N]
  __shared__ T Xs[kPhiK][kPhiT + 1];
  __shared__ T Ws[kPhiK][kPhiT];
  __shared__ int s_n;
  const int b = blockIdx.z, N = lat.N, Ne = lat.Ne, tid = threadIdx.x;
  if (vcfg && b >= *vcfg) return;  // whole CTA: past the valid configurations of a chunk
  const int8_t* ob = occ + (size_t)b * N;
  if (tid < 32) {  // one warp lists the occupied orbitals in order
    int n = 0;
    for (int base = 0; base < 2 * N; base += 32) {
      const int o = base + tid;
      const bool on = o < 2 * N && ((ob[o % N] >> (o / N)) & 1);
      const unsigned m = __ballot_sync(0xffffffffu, on);
      if (on) olist[n + __popc(m & ((1u << tid) - 1u))] = o;
      n += __popc(m);
    }
    if (tid == 0) s_n = n;
  }
  __syncthreads();
  double* P = phi + (size_t)b * Ne * Ne;
  const int k0 = blockIdx.y * kPhiT;
  // row tile -> spin and row range: tiles [0, tu) cover the up rows, the rest the down rows
  const int tu = (lat.n_up + kPhiT - 1) / kPhiT;
  const int s = (int)blockIdx.x < tu ? 0 : 1;
  const int r_lo = s == 0 ? 0 : lat.n_up, r_hi = s == 0 ? lat.n_up : Ne;
  const int a0 = r_lo + (s == 0 ? (int)blockIdx.x : (int)blockIdx.x - tu) * kPhiT;
  if (a0 >= r_hi || k0 >= Ne) return;  // whole CTA
  if ((err && *err) || s_n != Ne) {
    const double v = (err && *err) ? CUDART_NAN : 0.0;
    for (int q = tid; q < kPhiT * kPhiT; q += 256) {
      const int a = a0 + q / kPhiT, k = k0 + q % kPhiT;
      if (a < r_hi && k < Ne) P[(size_t)a * Ne + k] = v;
    }
    return;
  }
  const int tx = tid & 15, ty = tid >> 4;  // 4 columns x 4 rows each
  T acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = T(0);
  const T* W = net.proj_w + s * Ne;
  for (int kc = 0; kc < hl; kc += kPhiK) {
    for (int q = tid; q < kPhiK * kPhiT; q += 256) {  // X^T tile: channel kk of row r
      const int r = q / kPhiK, kk = q % kPhiK;
      const int a = a0 + r;
      T v = T(0);
      if (a < r_hi && kc + kk < hl) v = HL[((size_t)b * N + (olist[a] - s * N)) * hl + kc + kk];
      Xs[kk][r] = v;
    }
    for (int q = tid; q < kPhiK * kPhiT; q += 256) {  // W tile: channel kk, column k
      const int kk = q / kPhiT, c = q % kPhiT;
      Ws[kk][c] = (kc + kk < hl && k0 + c < Ne) ? W[(size_t)(kc + kk) * 2 * Ne + k0 + c] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kPhiK; ++kk) {
      T x[4], w[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) x[r] = Xs[kk][ty * 4 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) w[c] = Ws[kk][tx * 4 + c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] += x[r] * w[c];
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int a = a0 + ty * 4 + r;
    if (a >= r_hi) continue;
    const int o = olist[a];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int k = k0 + tx * 4 + c;
      if (k < Ne) P[(size_t)a * Ne + k] = (double)(net.M0[(size_t)o * Ne + k] + net.proj_b[s * Ne + k] + acc[r][c]);
    }
  }
}

// Tensor-core shape of a layer: n-tiles per warp and warps per row group, or 0.
struct MmaPlan {
  int ntw, wc;
};

MmaPlan plan_of(const scale_arch& a, int l) {
  const int ci = ace_width_in(a, l), co = ace_width_out(a, l);
  if (ci % 8 != 0) return {0, 0};
  if (l < a.n_conv) {
    if (a.family == SCALE_FAMILY_ACE) {  // conv block with the normalisation in the epilogue
      if (co == 48 || co == 144 || co == 192) return {co / 8, 1};
      return {0, 0};
    }
    if (co == 384) return {24, 2};  // wide SCALE conv (no normalisation)
    if (co == 640) return {20, 4};
    return {0, 0};
  }
  if (co == 64) return {8, 1};
  if (co == 128) return {16, 1};
  if (co == 256) return {16, 2};
  if (co == 512) return {16, 4};
  if (co == 1280) return {20, 8};
  return {0, 0};
}

size_t frag_layer_bytes(const scale_arch& a, int l) {
  const size_t taps = stencil_taps(a.stencil, a.ksize[l]);
  return taps * (size_t)ace_width_in(a, l) * ace_width_out(a, l) * 8;  // (ci/8)(co/8) 32 lanes x 16 B
}

template <int NTW, int WC, bool LN>
void run_mma(cudaStream_t st, const Lattice& lat, const WFrag* frag, const float* bias, const float* g,
             const float* be, int ks, int stencil, int cin, int res, int act, float eps, const float* in,
             float* out, long long rows, const int* vcfg) {
  constexpr int ROWS = 16 * (8 / WC);
  const long long blocks = (rows + ROWS - 1) / ROWS;
  k_ace_mma<NTW, WC, LN><<<(unsigned)blocks, 256, 0, st>>>(lat, frag, bias, g, be, ks, stencil, cin, res, act, eps,
                                                            in, out, rows, vcfg);
}

bool launch_mma_layer(cudaStream_t st, const Lattice& lat, const MmaPlan& p, bool ln, const WFrag* frag,
                      const float* bias, const float* g, const float* be, int ks, int stencil, int cin, int res,
                      int act, float eps, const float* in, float* out, long long rows, const int* vcfg) {
#define SCALE_ACE_MMA(NTW, WC, LN) \
  run_mma<NTW, WC, LN>(st, lat, frag, bias, g, be, ks, stencil, cin, res, act, eps, in, out, rows, vcfg)
  if (ln) {
    if (p.ntw == 6) SCALE_ACE_MMA(6, 1, true);
    else if (p.ntw == 18) SCALE_ACE_MMA(18, 1, true);
    else if (p.ntw == 24) SCALE_ACE_MMA(24, 1, true);
    else return false;
  } else {
    if (p.ntw == 8 && p.wc == 1) SCALE_ACE_MMA(8, 1, false);
    else if (p.ntw == 16 && p.wc == 1) SCALE_ACE_MMA(16, 1, false);
    else if (p.ntw == 16 && p.wc == 2) SCALE_ACE_MMA(16, 2, false);
    else if (p.ntw == 16 && p.wc == 4) SCALE_ACE_MMA(16, 4, false);
    else if (p.ntw == 20 && p.wc == 4) SCALE_ACE_MMA(20, 4, false);
    else if (p.ntw == 20 && p.wc == 8) SCALE_ACE_MMA(20, 8, false);
    else if (p.ntw == 24 && p.wc == 2) SCALE_ACE_MMA(24, 2, false);
    else return false;
  }
#undef SCALE_ACE_MMA
  return true;
}

// Layers that run on tcgen05 when the tensor-core path is on: the conv layers (checked at
// creation), then the site-wise layers up to the first one of an unsupported shape. Between
// two of them the activations stay split (hi, lo); the rest run on the mma.sync kernels.
bool tc_layer(const scale_ctx* c, int l) {
  if (!c->ace_tc) return false;
  for (int j = c->arch.n_conv; j <= l; ++j)
    if (!tc_sitewise(ace_width_in(c->arch, j), ace_width_out(c->arch, j)) || c->arch.residual[j]) return false;
  return true;
}

// Layers [l0, l1) on `rows` rows: a holds the input of layer l0 (as (hi, lo) halves of the
// buffer when split), b is the other buffer; on return *out points at the buffer holding the
// output of layer l1 - 1 and *out_split tells whether it is split. Rows are the sites of
// configurations of lat (rows = configurations x lat.N); the site-wise (1 x 1) layers read
// row r alone, so they also run on a buffer of gathered rows whose lattice is a stand-in.
template <typename T>
cudaError_t ace_layers_t(scale_ctx* c, const Lattice& lat, int l0, int l1, T* a, T* b, long long rows, bool split,
                         const int* vcfg, T** out, bool* out_split) {
  const AceNet<T> net = make_ace_net<T>(c);
  size_t frag_off = 0;
  for (int l = 0; l < l0; ++l) frag_off += frag_layer_bytes(c->arch, l);
  for (int l = l0; l < l1; ++l) {
    bool done = false;
    if constexpr (sizeof(T) == 4) {
      if (split && tc_layer(c, l)) {  // on tcgen05; split output when the next layer is too
        const float* bimg = (const float*)((const char*)c->ace_frag + frag_off);
        const long long tin = rows * net.cin[l], tout = rows * net.cout[l];
        float* olo = (l + 1 < l1 && tc_layer(c, l + 1)) ? b + tout : nullptr;
        const cudaError_t e =
            launch_conv_tc(c, lat, net.ln_g[l] != nullptr, net.cin[l], net.cout[l], c->arch.residual[l], net.ks[l],
                           bimg, net.bias[l], net.ln_g[l], net.ln_b[l], net.act, (float)net.eps, a, a + tin, b, olo,
                           rows, vcfg);
        if (e != cudaSuccess) return e;
        split = olo != nullptr;
        done = true;
      } else if (c->ace_mma) {
        const MmaPlan p = plan_of(c->arch, l);
        const WFrag* frag = (const WFrag*)((const char*)c->ace_frag + frag_off);
        done = launch_mma_layer(c->stream, lat, p, net.ln_g[l] != nullptr, frag, net.bias[l], net.ln_g[l],
                                net.ln_b[l], net.ks[l], net.stencil, net.cin[l], c->arch.residual[l], net.act,
                                (float)net.eps, a, b, rows, vcfg);
      }
    }
    if (!done) {
      const long long blocks = (rows + kAceRowsGeneric - 1) / kAceRowsGeneric;
      k_ace_layer<T><<<(unsigned)blocks, 32 * kAceRowsGeneric, 0, c->stream>>>(
          lat, net.kernel[l], net.bias[l], net.ln_g[l], net.ln_b[l], net.ks[l], net.stencil, net.cin[l],
          net.cout[l], c->arch.residual[l], net.act, net.eps, a, b, rows, vcfg);
    }
    frag_off += frag_layer_bytes(c->arch, l);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    std::swap(a, b);
  }
  *out = a;
  *out_split = split;
  return cudaSuccess;
}

template <typename T>
cudaError_t ace_forward_t(scale_ctx* c, const int8_t* occ, int C, double* phi64, const int* vcfg, void* hl_out) {
  const AceNet<T> net = make_ace_net<T>(c);
  const int N = c->N;
  const long long rows = (long long)C * N;
  T* a = (T*)c->act_a;
  T* b = (T*)c->act_b;
  const long long total = rows * c->h;
  const int eblocks = (int)std::min<long long>((total + 255) / 256, 152LL * 64);
  bool split = false;  // activations held as (hi, lo) halves of the buffer
  if constexpr (sizeof(T) == 4) {
    if (c->ace_tc) {
      k_ace_embed_split<<<eblocks, 256, 0, c->stream>>>(N, c->h, net.per_site, net.embed, occ, total, a,
                                                        a + total, vcfg);
      split = true;
    }
  }
  if (!split) k_ace_embed<T><<<eblocks, 256, 0, c->stream>>>(N, c->h, net.per_site, net.embed, occ, total, a, vcfg);
  T* hL = nullptr;
  bool hsplit = false;
  cudaError_t e = ace_layers_t<T>(c, c->lat, 0, c->L, a, b, rows, split, vcfg, &hL, &hsplit);
  if (e != cudaSuccess) return e;
  const int hl = net.cout[c->L - 1];
  if (hl_out) {  // the last layer's features (plain rows: the last layer never writes a split)
    e = cudaMemcpyAsync(hl_out, hL, sizeof(T) * (size_t)rows * hl, cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return e;
  }
  const int Ne = c->Ne;
  const dim3 pgrid((c->sys.n_up + kPhiT - 1) / kPhiT + (c->sys.n_dn + kPhiT - 1) / kPhiT, (Ne + kPhiT - 1) / kPhiT, C);
  e = cudaFuncSetAttribute(k_ace_phi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(int) * 2 * N));
  if (e != cudaSuccess) return e;
  k_ace_phi<T><<<pgrid, 256, sizeof(int) * 2 * N, c->stream>>>(c->lat, net, hl, occ, hL, c->ace_err, phi64, vcfg);
  return cudaGetLastError();
}

}  // namespace

bool ace_tc_shapes(const scale_arch& a) {
  if (a.family == SCALE_FAMILY_ACE) {
    if (a.stencil != SCALE_STENCIL_BOX || !tc_width(a.h)) return false;
    for (int l = 0; l < a.n_conv; ++l)
      if (a.ksize[l] != 3) return false;
    return ace_mma_shapes(a);
  }
  if (a.family == SCALE_FAMILY_WIDE) {  // one conv: 3x3 box or 5x5 plus, then site-wise layers
    if (a.n_conv != 1 || !tc_wide_width(a.h)) return false;
    const bool box3 = a.ksize[0] == 3 && a.stencil == SCALE_STENCIL_BOX;
    const bool plus5 = a.ksize[0] == 5 && a.stencil == SCALE_STENCIL_DISK;
    return (box3 || plus5) && ace_mma_shapes(a);
  }
  return false;
}

bool ace_mma_shapes(const scale_arch& a) {
  for (int l = 0; l < a.n_layers; ++l)
    if (plan_of(a, l).ntw == 0) return false;
  return true;
}

size_t ace_frag_bytes(const scale_arch& a) {
  if (!ace_mma_shapes(a)) return 0;
  size_t t = 0;
  for (int l = 0; l < a.n_layers; ++l) t += frag_layer_bytes(a, l);
  return t;
}

cudaError_t launch_ace_build(scale_ctx* c) {
  if (!c->ace_mma) return cudaSuccess;
  const AceNet<float> net = make_ace_net<float>(c);
  size_t off = 0;
  for (int l = 0; l < c->L; ++l) {
    const int taps = stencil_taps(net.stencil, net.ks[l]);
    if (tc_layer(c, l)) {  // the tcgen05 weight-tile image
      const size_t n = (size_t)taps * 2 * net.cin[l] * net.cout[l];
      const int blocks = (int)std::min<size_t>((n + 255) / 256, 4096);
      k_ace_build_bimg<<<blocks, 256, 0, c->stream>>>(net.kernel[l], net.cin[l], net.cout[l], taps,
                                                       (float*)((char*)c->ace_frag + off));
      off += frag_layer_bytes(c->arch, l);
      continue;
    }
    const size_t n = (size_t)taps * (net.cin[l] / 8) * (net.cout[l] / 8) * 32;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 4096);
    k_ace_build_frag<<<blocks, 256, 0, c->stream>>>(net.kernel[l], taps, net.cin[l], net.cout[l],
                                                     (WFrag*)((char*)c->ace_frag + off));
    off += frag_layer_bytes(c->arch, l);
  }
  return cudaGetLastError();
}

// Slater matrices (FP64) of C configurations occ[C][N] through the ACE network; the
// activations go to the context's scratch buffers. vcfg (optional, device): only the first
// *vcfg configurations are evaluated (the rest of the launch returns at once).
cudaError_t launch_ace_forward(scale_ctx* c, const int8_t* occ, int C, double* phi64, const int* vcfg,
                               void* hl_out) {
  if (C <= 0) return cudaSuccess;
  if (c->fp64) return ace_forward_t<double>(c, occ, C, phi64, vcfg, hl_out);
  return ace_forward_t<float>(c, occ, C, phi64, vcfg, hl_out);
}

// Layers [l0, l1) on a buffer of rows (see ace_layers_t); *out receives the buffer of the
// last output.
cudaError_t launch_ace_layers(scale_ctx* c, const Lattice& lat, int l0, int l1, void* a, void* b, long long rows,
                              bool split, const int* vcfg, void** out) {
  bool os = false;
  if (c->fp64) return ace_layers_t<double>(c, lat, l0, l1, (double*)a, (double*)b, rows, false, vcfg, (double**)out, &os);
  return ace_layers_t<float>(c, lat, l0, l1, (float*)a, (float*)b, rows, split, vcfg, (float**)out, &os);
}

bool ace_tc_layer(const scale_ctx* c, int l) { return tc_layer(c, l); }

}  // namespace scale
