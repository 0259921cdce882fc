// scale_internal.cuh -- shared declarations of the SCALE CUDA library (sm_103a).
//
// Data layout in HBM (per context, B = loaded samples, T = double in FP64 mode, float in
// mixed mode):
//   occ          int8  [B][N]            local states 0,1,2,3
//   orb_of_slot  int32 [B][Ne]           orbital o = s*N + i held by each determinant row
//   slot_of_orb  int32 [B][2N]           inverse map, -1 when the orbital is empty
//   z0           T     [B][N][h]         pre-activation of layer 0 (kept for the additive
//                                        receptive-field update of Eq. neighbor)
//   HL           T     [B][N][h]         last-layer features H(L)
//   Binv         T     [B][Ne][Ne]       Binv[c][k] = (Phi^-1)[k][c]: row c is the dual
//                                        vector of determinant row c (M[o_a] . Binv[c] = delta)
//   Pt           T     [B][2][Ne][h]     Pt[s][c] = W_s Binv[c], W_s = proj_w[:, s*Ne:(s+1)*Ne]
//   logabs       f64   [B]               log|det Phi| in slot order, sign_slot int32 [B]
// Parameters are kept as FP64 and T copies; the layer-0 conv-of-embedding table
//   KE [Ns][4][taps0][h] = K_0[d]^T E_t[n]   (Ns = N with per-site tables, else 1; d over the
//                                             taps of layer 0's stencil)
// turns the layer-0 receptive-field update into table additions.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/scale.h"

namespace scale {

constexpr int kMaxLayers = SCALE_MAX_LAYERS;
constexpr int kMaxH = 64;

// Lattice geometry and Hamiltonian constants, passed by value to kernels.
struct Lattice {
  int Lx, Ly, pbc_x, pbc_y, N, n_up, n_dn, Ne, model;
  double t, tp, U, J;
};

// Elements of one sample's commit scratch: the matrix D and the saved Binv rows ([32][NeP]
// each, NeP = Ne rounded up to 4; 32 = the largest rank r) and the saved G0t rows ([32][2N]).
__host__ __device__ inline size_t commit_scratch_elems(int Ne, int N) {
  return (size_t)2 * 32 * ((Ne + 3) & ~3) + (size_t)32 * 2 * N;
}

// Offset (dx, dy) of tap d of a k x k layer: taps run over the box in row-major order; the
// disk stencil keeps the offsets within L2 distance (k-1)/2 (k = 5: the 13 sites of SCALE-L).
__host__ __device__ __forceinline__ void stencil_tap(int stencil, int k, int d, int& dx, int& dy) {
  const int r = (k - 1) / 2;
  if (stencil == SCALE_STENCIL_BOX) {
    dx = d % k - r;
    dy = d / k - r;
    return;
  }
  int t = 0;
  for (int q = 0; q < k * k; ++q) {
    const int x = q % k - r, y = q / k - r;
    if (x * x + y * y > r * r) continue;
    if (t == d) {
      dx = x;
      dy = y;
      return;
    }
    ++t;
  }
  dx = dy = 0;
}

__host__ __device__ __forceinline__ bool stencil_in(int stencil, int k, int dx, int dy) {
  const int r = (k - 1) / 2;
  return stencil == SCALE_STENCIL_BOX || dx * dx + dy * dy <= r * r;
}

// Site reached from i by (dx, dy), or -1 past an open edge.
__host__ __device__ __forceinline__ int site_off(const Lattice& lat, int i, int dx, int dy) {
  int x = i % lat.Lx + dx, y = i / lat.Lx + dy;
  if (x < 0 || x >= lat.Lx) {
    if (!lat.pbc_x) return -1;
    x = ((x % lat.Lx) + lat.Lx) % lat.Lx;
  }
  if (y < 0 || y >= lat.Ly) {
    if (!lat.pbc_y) return -1;
    y = ((y % lat.Ly) + lat.Ly) % lat.Ly;
  }
  return y * lat.Lx + x;
}

// Network parameters in precision T (device pointers).
template <typename T>
struct Net {
  int h, L, act, per_site;
  int stencil;                   // SCALE_STENCIL_* of the k x k layers
  int taps0;                     // taps of layer 0 under the stencil
  int ksize[kMaxLayers];
  int resid[kMaxLayers];
  const T* embed;                // [Ns][4][h]
  const T* kernel[kMaxLayers];   // [k][k][h][h]
  const T* bias[kMaxLayers];     // [h]
  const T* proj_w;               // [h][2Ne]
  const T* proj_b;               // [2Ne]
  const T* M0;                   // [2N][Ne]
  const T* M0b;                  // [2N][Ne] M0[o] + proj_b[s(o)] (derived at set_params)
  const T* KE;                   // [Ns][4][taps0][h]
};

// FP32 tanh for the tensor-core layers. For |z| < 1/2, tanh z = z + z s q(s) with s = z^2 and
// q the cubic that minimises the largest relative error on (0, 1/2] (1.5e-8, below the FP32
// rounding; fitted by fit_tanh_poly.py beside this file: tanh z = z - z^3/3 + 2z^5/15 - ...,
// so q(0) = -1/3); above, tanh|z| = (1 - e^{-2|z|}) / (1 + e^{-2|z|}) (no cancellation once
// |z| >= 1/2).
__device__ __forceinline__ float tanh_f32_small(float z) {  // |z| < 1/2
  const float s = z * z;
  float p = 1.724151708e-02f;
  p = fmaf(p, s, -5.304550752e-02f);
  p = fmaf(p, s, 1.332587898e-01f);
  p = fmaf(p, s, -3.333314359e-01f);
  return fmaf(z * s, p, z);
}
__device__ __forceinline__ float tanh_f32(float z) {
  const float a = fabsf(z);
  const float small = tanh_f32_small(z);
  float e;  // e^{-2|z|} = 2^{|z| (-2 log2 e)}, one multiply into the hardware base-2 exponential
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(a * -2.8853900817779268f));
  const float big = copysignf(__fdividef(1.f - e, 1.f + e), z);
  return a < 0.5f ? small : big;
}

template <typename T>
__device__ __forceinline__ T act_fn(int act, T z) {
  if (act == SCALE_ACT_TANH) return tanh(z);
  return z / (T(1) + exp(-z));
}
// Activation of the tensor-core layers (FP32): own tanh, SiLU through the FP32 exp.
__device__ __forceinline__ float act_fast(int act, float z) {
  if (act == SCALE_ACT_TANH) return tanh_f32(z);
  return z / (1.f + __expf(-z));
}

template <typename T>
__device__ __forceinline__ T act_grad(int act, T z) {
  if (act == SCALE_ACT_TANH) {
    T th = tanh(z);
    return T(1) - th * th;
  }
  T s = T(1) / (T(1) + exp(-z));
  return s * (T(1) + z * (T(1) - s));
}

}  // namespace scale

// The context (opaque to callers).
struct scale_ctx {
  scale_system sys;
  scale_arch arch;
  scale::Lattice lat;
  int N = 0, Ne = 0, h = 0, L = 0, k0 = 1, r0 = 0;
  bool fp64 = true;
  bool lowrank_ok = false;  // SCALE layer layout (k_l = 1 for l >= 1)
  bool use_mma = false;     // mixed mode, SCALE layout, h in {16, 32, 64}: site-wise layers on tensor cores
  void* et_wimg = nullptr;  // batched tensor-core local energies (eloc_tc.cu): weight image, or null
  int et_rows = 0;          // rows per move slot of that kernel (largest affected set)
  int et_inject = 0;        // test hook: leave the next launch's first hand-off unsignalled
  int hpad = 16;            // channel capacity of the per-warp scratch (16, 32 or 64)
  void* wfrag = nullptr;    // hi/lo mma fragments (TF32, or BF16 as an option) of the site-wise layers
  int64_t P = 0;
  int B_max = 0, B = 0;
  int max_moves = 0;
  cudaStream_t stream = nullptr;
  size_t budget = 0, allocated = 0;
  std::string err;
  bool params_set = false;

  // parameters
  double* params64 = nullptr;
  float* params32 = nullptr;
  double* M0_64 = nullptr;
  float* M0_32 = nullptr;
  void* M0b = nullptr;  // [2N][Ne] T: M0[o] + proj_b[s(o)]
  void* KE = nullptr;

  // lattice tables
  int32_t* bonds = nullptr;  // [nb_nn + nb_nnn][2]
  int nb_nn = 0, nb_nnn = 0;

  // per-sample state
  int8_t* occ = nullptr;
  int32_t* orb_of_slot = nullptr;
  int32_t* slot_of_orb = nullptr;
  void* z0 = nullptr;
  void* HL = nullptr;
  void* Binv = nullptr;
  void* Pt = nullptr;
  void* G0t = nullptr;  // [B][Ne][2N] T: G0t[j][o] = (M0[o] + proj_b[s(o)]) . Binv[j]
  double* logabs = nullptr;
  int32_t* sign_slot = nullptr;
  int32_t* status = nullptr;
  int32_t* commits = nullptr;
  double* drift = nullptr;

  // scratch
  double* Phi64 = nullptr;     // [B][Ne][Ne]
  void* act_a = nullptr;       // [B][N][h]
  void* act_b = nullptr;       // [B][N][h]
  int32_t* list = nullptr;     // [B] sample list for partial refresh
  int32_t* list_count = nullptr;
  double* stat_dev = nullptr;  // [4]: drift maximum (bits), then int32 commits, refreshes, drift refreshes
  void* commit_scratch = nullptr;  // [B][3*32*Ne + 2*32*kMaxH] T
  double* la_tmp = nullptr;     // [B] log|psi| scratch (ascending)
  int32_t* sg_tmp = nullptr;    // [B]
  double* full_la = nullptr;    // [FC] chunk determinants (FC = max(max_batch, full_chunk))
  int32_t* full_sg = nullptr;   // [FC]
  double* full_diag = nullptr;  // [B]
  int64_t* full_offsets = nullptr;  // [B+1] device copy of the packed offsets
  void* grad_scratch = nullptr;
  size_t grad_scratch_bytes = 0;
  int32_t* move_count = nullptr;  // [B] connected configurations last enumerated

  // full-recompute path scratch (a chunk is full_chunk configurations, sized from memory and
  // not from max_batch; the chunk buffers hold FC = max(max_batch, full_chunk) entries)
  int full_chunk = 0;
  int8_t* full_occ = nullptr;      // [FC][N]
  int32_t* full_owner = nullptr;   // [FC] entry index b * (max_moves + 1) + m, or -1
  int32_t* full_list = nullptr;    // [FC] g for a valid chunk position, -1 past the total
  int32_t* full_vcount = nullptr;  // [1] valid positions of the current chunk
  double* full_coeff = nullptr;    // [B][max_moves]
  int32_t* full_moves = nullptr;   // [B][max_moves][4]
  double* full_la_all = nullptr;   // [B][max_moves + 1] log|psi| of n (m = 0) and its n'
  int32_t* full_sg_all = nullptr;  // [B][max_moves + 1]

  // ACE family (full-recompute network, no cached update)
  bool ace = false;
  bool ace_mma = false;     // mixed mode with tensor-core shapes for every layer
  bool ace_tc = false;      // conv blocks on tcgen05 (widths 48, 144, 192)
  int32_t* ace_err = nullptr;  // set by a tcgen05 layer whose bounded wait ran out
  int hmax = 0;             // widest layer (activation buffers are [B][N][hmax])
  void* ace_frag = nullptr; // TF32 hi/lo mma fragments of every ACE layer

  // cached update at the wide SCALE shapes (wide_lowrank.cu): the caches z0 [B][N][h],
  // HL [B][N][h_last], Binv and Pt [B][2][Ne][h_last] above, and per chunk of moves
  bool wide_lr = false;
  int wl_rows = 0;            // row slots per move: the largest affected set of any move
  int wl_chunk = 0;           // moves per chunk (their rows fill the activation buffers)
  void* wl_meta = nullptr;    // [wl_chunk] per-move record of the chunk

  scale_stats stats{};
};

namespace scale {

// ACE widths: the conv blocks keep h, the site-wise layers after them have h_mlp.
constexpr int kAceMaxH = 256;
constexpr int kAceMaxHMlp = 512;
constexpr int kWideMaxH = 1024;
constexpr int kWideMaxHMlp = 2048;
inline int ace_width_out(const scale_arch& a, int l) {
  return l < a.n_conv ? a.h : (a.h_mlp > 0 ? a.h_mlp : a.h);
}
// Taps of a k x k layer under the network's stencil (row-major box order).
__host__ __device__ inline bool stencil_has(int stencil, int k, int dx, int dy) {
  const int r = (k - 1) / 2;
  return stencil == SCALE_STENCIL_BOX || dx * dx + dy * dy <= r * r;
}
inline int stencil_taps(int stencil, int k) {
  int n = 0;
  for (int dy = -(k - 1) / 2; dy <= (k - 1) / 2; ++dy)
    for (int dx = -(k - 1) / 2; dx <= (k - 1) / 2; ++dx) n += stencil_has(stencil, k, dx, dy);
  return n;
}
inline int ace_width_in(const scale_arch& a, int l) { return l == 0 ? a.h : ace_width_out(a, l - 1); }
// Bytes of the tensor-core fragments of every ACE layer (0 when a shape has none).
size_t ace_frag_bytes(const scale_arch& a);
bool ace_mma_shapes(const scale_arch& a);
bool ace_tc_shapes(const scale_arch& a);
cudaError_t launch_ace_build(scale_ctx* c);
cudaError_t launch_ace_forward(scale_ctx* c, const int8_t* occ, int C, double* phi64, const int* vcfg = nullptr,
                               void* hl_out = nullptr);
cudaError_t launch_ace_layers(scale_ctx* c, const Lattice& lat, int l0, int l1, void* a, void* b, long long rows,
                              bool split, const int* vcfg, void** out);
bool ace_tc_layer(const scale_ctx* c, int l);

// cached update at the wide SCALE shapes (wide_lowrank.cu)
bool wide_lowrank_shapes(const scale_arch& a);
int wide_rows_per_move(const scale_system& s, const scale_arch& a);
size_t wide_meta_bytes();
cudaError_t launch_wide_params(scale_ctx* c);
cudaError_t launch_wide_cache(scale_ctx* c, int B);
cudaError_t launch_wide_eloc(scale_ctx* c, double* eloc);
// exclusive prefix sums offsets[b] = sum_{b' < b} (count[b'] + extra), offsets[B] = total
cudaError_t launch_offsets(scale_ctx* c, int B, const int32_t* count, int extra, int64_t* offsets);

// kernels (launch wrappers), each enqueued on ctx->stream
// count (optional, device): sample_list is compacted, its first *count entries are used
cudaError_t launch_forward(scale_ctx* c, const int8_t* occ, int B, const int32_t* sample_list,
                           bool keep_cache, double* phi_out, const int32_t* count = nullptr);
cudaError_t launch_slots(scale_ctx* c, const int8_t* occ, int B);
cudaError_t launch_gj(scale_ctx* c, const double* Phi, int n, int B, const int32_t* list,
                      bool inverse, bool out_fp64, void* Binv, double* logabs, int32_t* sign,
                      int32_t* status);
cudaError_t launch_projector(scale_ctx* c, int B, const int32_t* list, const int32_t* count = nullptr);
// G0t = (M0 + proj_b) Binv^T of the listed samples (all B when list is null).
cudaError_t launch_build_g0(scale_ctx* c, int B, const int32_t* list, const int32_t* count = nullptr);
cudaError_t launch_build_ke(scale_ctx* c);
cudaError_t launch_build_wfrag(scale_ctx* c);
cudaError_t launch_eloc_lowrank_list(scale_ctx* c, const int32_t* list, int n, double* eloc);
cudaError_t launch_logpsi_list(scale_ctx* c, const int32_t* list, int n, double* logabs, int32_t* sign);
cudaError_t launch_load_list(scale_ctx* c, const int8_t* occ, const int32_t* list, int n);
cudaError_t launch_logpsi_out(scale_ctx* c, double* logabs, int32_t* sign);
cudaError_t launch_eloc_lowrank(scale_ctx* c, double* eloc);
cudaError_t launch_ratios(scale_ctx* c, const int32_t* moves, int M, double* ratio);
cudaError_t launch_commit(scale_ctx* c, const int32_t* moves);
cudaError_t launch_metropolis(scale_ctx* c, const int32_t* pick, const int32_t* dir, const double* u,
                              int32_t* accepted);
cudaError_t launch_log_psi_sym(scale_ctx* c, int G, const int32_t* perms, const double* chi, double* logabs,
                               int32_t* sign);
cudaError_t launch_eloc_full(scale_ctx* c, double* eloc);
cudaError_t launch_grad(scale_ctx* c, double* grad, int recompute);
cudaError_t refresh_samples(scale_ctx* c, bool force_all, bool counters_due = true);
cudaError_t launch_mark_refresh(scale_ctx* c, bool force_all, bool counters_due);
cudaError_t launch_slots_list(scale_ctx* c, const int32_t* list, int B);
cudaError_t launch_forward_phi(scale_ctx* c, const int8_t* occ, int B, const int32_t* list, const int32_t* vcount,
                               double* phi);

template <typename T>
Net<T> make_net(scale_ctx* c);

// batched tensor-core local energies (eloc_tc.cu)
int et_rows_per_move(const scale_ctx* c, const std::vector<int32_t>& bonds);
size_t et_wimg_bytes(const scale_ctx* c);
bool et_supported(const scale_ctx* c, int rows_per_move, int smem_optin);
cudaError_t launch_build_et(scale_ctx* c);
cudaError_t launch_eloc_tc(scale_ctx* c, double* eloc, const int32_t* list, int n);

}  // namespace scale
