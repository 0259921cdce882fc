// eloc_tc.cu -- local energies of the cached update (Sec. II.C: Eq. neighbor, Eq. SMW) with the
// site-wise layers (Eq. MLP) of all connected configurations batched onto the 5th-generation
// tensor cores. Mixed precision, 32 channels.
//
// One CTA of 16 warps per walker. The warps take two roles and hand batches of moves to each
// other through shared memory and mbarriers:
//   move warps (12): for each move of a batch, the affected sites S (Eq. neighbor) and the
//     layer-0 output rows  x_s = E_s[n'_s] + act(z0_s + sum of layer-0 table deltas)  in the
//     move's slot of a batch buffer (one row per site of S); once the site-wise layers have
//     run, the rank-r matrix R of Eq. SMW from the new features H'(L), the projector
//     Pt = W Phi^-1 and the cached inverse, and det R;
//   MLP warps (4): the site-wise layers on the batch's 256 rows (two MMA tiles of 128 rows):
//     tcgen05.mma kind::tf32 with the activations as the A operand in Tensor Memory (hi and lo
//     halves of a TF32 split), each layer's hi/lo weight tiles as the B operand in shared
//     memory, three products per K step (hi*hi + lo*hi + hi*lo) accumulated in FP32 in TMEM,
//     and the epilogue (bias, activation, split of the next layer's input) in registers with
//     one thread per row.
// Two batch buffers alternate: the move warps stage batch g+1 and finish batch g-1 while the
// MLP warps run batch g. The contribution of every move is stored by its enumeration index and
// the chunk's sum is taken in that order, so E_loc does not depend on the scheduling.
//
// Every wait is bounded; a wait that runs out sets the kernel's error word, the walker's
// E_loc becomes NaN, outstanding MMAs are awaited (bounded) and TMEM is released.
#include <algorithm>
#include <vector>

#include "eloc_common.cuh"
#include "tcgen05.cuh"

namespace scale {

namespace {

constexpr int kEtH = 32;                 // channels
constexpr int kEtLd = kEtH + 4;          // row stride of the batch buffers (floats)
constexpr int kEtMlpWarps = 4;        // one per TMEM lane quarter: thread = row, all channels
constexpr int kEtCols = kEtH * 4 / kEtMlpWarps;  // channels of a row per MLP thread
constexpr int kEtWork = 12;
constexpr int kEtWarps = kEtMlpWarps + kEtWork;
constexpr int kEtThreads = 32 * kEtWarps;
constexpr int kEtRows = 256;             // rows of a batch: two MMA tiles
constexpr int kEtMaxMoves = 64;          // moves of a batch at most
constexpr int kEtTileCols = 3 * kEtH;    // TMEM columns of one MMA tile: D, A hi, A lo
constexpr int kEtTmemCols = 256;         // allocation (power of two >= 2 * kEtTileCols)
constexpr int kEtKT = kEtH / 8;          // K steps of one layer
constexpr uint32_t kEtPolls = 1u << 20;  // bound of every mbarrier wait (a batch takes microseconds)
constexpr uint32_t kEtIdesc = tc::idesc_tf32<128, kEtH>();

// One move of a batch, written by its move warp when it stages the move.
struct EtMeta {
  int16_t site[kSMax];
  int8_t nold[kSMax], nnew[kSMax];
  int nS;
};

// Per move warp: the rank-r matrix and the electron list of its current move.
struct EtScratch {
  float R[kRMax][kRMax + 1];
  int slot[kRMax], orb[kRMax], sidx[kRMax], moved[kRMax];
};

// Dynamic shared memory, in bytes from a 128-byte aligned base.
struct EtLayout {
  size_t wimg, bbuf, meta, scr, mlist, contrib, slot, occ, total;
  __host__ __device__ EtLayout(int nsw, int N) {
    size_t o = 0;
    wimg = o;  // [nsw][KT][hi, lo][H x 8] B tiles
    o += (size_t)nsw * 2 * kEtH * kEtH * 4;
    bbuf = o;  // [2][kEtRows][kEtLd]
    o += (size_t)2 * kEtRows * kEtLd * 4;
    meta = o;  // [2][kEtMaxMoves]
    o += (size_t)2 * kEtMaxMoves * sizeof(EtMeta);
    o = (o + 15) & ~(size_t)15;
    scr = o;  // [kEtWork]
    o += (size_t)kEtWork * sizeof(EtScratch);
    mlist = o;
    o += (size_t)kMoveChunk * 4;
    contrib = o;
    o += (size_t)kMoveChunk * 8;
    slot = o;
    o += (size_t)2 * N * 4;
    occ = o;
    o += (size_t)N;
    total = (o + 15) & ~(size_t)15;
  }
};

struct EtArgs {
  const float* wimg;  // weight image (global), copied to shared memory by every CTA
  int nsw;            // site-wise layers (L - 1)
  int rpm;            // rows per move slot: the largest affected set of any move
  int mb;             // moves per batch
  int* err;           // set when a bounded wait ran out
  int inject;         // test hook: the first batch's hand-off to the MLP warps is not signalled
};

// Byte offset of element (n, k) of an [N x 8] tf32 tile in the K-major core-matrix layout
// without swizzle: core matrix (n / 8, k / 4) at ((n / 8) * 2 + k / 4) * 128 bytes, its row
// n % 8 at 16 bytes; core matrices adjacent along K are 128 bytes apart (descriptor LBO),
// along N 256 bytes (SBO).
__host__ __device__ constexpr uint32_t et_off(int n, int k) {
  return (uint32_t)(((n >> 3) * 2 + (k >> 2)) * 128 + (n & 7) * 16 + (k & 3) * 4);
}

// Weight image of the site-wise layers l = 1..L-1: tile (l-1, kk, hl) holds the hi (hl = 0) or
// lo (hl = 1) TF32 half of B[n][k] = W_l[8 kk + k][n] (the MMA computes D = A B^T).
__global__ void k_build_et_wimg(Net<float> net, int nsw, float* __restrict__ out) {
  const int per_tile = kEtH * 8;
  const int total = nsw * kEtKT * 2 * per_tile;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const int e = q % per_tile, tile = q / per_tile;
    const int hl = tile & 1, kk = (tile >> 1) % kEtKT, l = (tile >> 1) / kEtKT + 1;
    const int n = e / 8, k = e % 8;
    const float w = net.kernel[l][(size_t)(8 * kk + k) * kEtH + n];
    uint32_t hi, lo;
    split_tf32(w, hi, lo);
    out[(size_t)tile * per_tile + et_off(n, k) / 4] = __uint_as_float(hl ? lo : hi);
  }
}

// Activation of 16 values of a thread. tanh: when every |z| of the warp is below 0.5 (the
// usual case) only the series branch of tanh_f32 is evaluated; the result is the same.
template <int NV>
__device__ __forceinline__ void et_act(int act, float (&z)[NV]) {
  if (act == SCALE_ACT_TANH) {
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < NV; ++j) m = fmaxf(m, fabsf(z[j]));
    if (__all_sync(0xffffffffu, m < 0.5f)) {
#pragma unroll
      for (int j = 0; j < NV; ++j) z[j] = tanh_f32_small(z[j]);
    } else {
#pragma unroll
      for (int j = 0; j < NV; ++j) z[j] = tanh_f32(z[j]);
    }
  } else {
#pragma unroll
    for (int j = 0; j < NV; ++j) z[j] = act_fast(act, z[j]);
  }
}

// Split NV values into TF32 hi and lo halves and store them to consecutive TMEM columns from
// hi_addr and lo_addr, for the warp's 32 lanes (no wait).
template <int NV>
__device__ __forceinline__ void et_store_split(uint32_t hi_addr, uint32_t lo_addr, const float (&x)[NV]) {
#pragma unroll
  for (int h8 = 0; h8 < NV / 8; ++h8) {
    uint32_t hi[8], lo[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) split_tf32(x[8 * h8 + j], hi[j], lo[j]);
    tc::tmem_st8(hi_addr + 8 * h8, hi);
    tc::tmem_st8(lo_addr + 8 * h8, lo);
  }
}

// Determinant of R (r <= 16): lane i holds row i in registers; each step takes the largest
// |value| of column k among the unused rows (ties to the lowest row) as pivot, broadcasts its
// row and eliminates column k from the other unused rows. The rows are never swapped; the sign
// of the pivot order is the parity of the unused rows below each pivot. The steps are expanded
// by template recursion so that every register index is a compile-time constant.
struct EtLu {
  float det;
  int parity;
  unsigned unused;
  bool zero;
};

template <int K>
__device__ __forceinline__ void et_lu_step(float (&v)[16], int r, EtLu& st) {
  if (K < r && !st.zero) {  // uniform
    const int lane = threadIdx.x & 31;
    const bool cand = (st.unused >> lane) & 1u;
    const unsigned key = cand ? __float_as_uint(fabsf(v[K])) : 0u;
    const unsigned mx = __reduce_max_sync(0xffffffffu, key);
    st.zero = mx == 0u;  // column K vanishes on every unused row
    const int p = (__ffs(__ballot_sync(0xffffffffu, cand && key == mx)) - 1) & 31;
    const float pv = __shfl_sync(0xffffffffu, v[K], p);
    st.det *= pv;
    st.parity ^= __popc(st.unused & ((1u << p) - 1u)) & 1;
    st.unused &= ~(1u << p);
    const bool upd = (st.unused >> lane) & 1u;
    const float f = upd ? v[K] * recip(pv) : 0.f;
#pragma unroll
    for (int j = K + 1; j < 16; ++j) {
      const float pj = __shfl_sync(0xffffffffu, v[j], p);
      if (upd) v[j] = fmaf(-f, pj, v[j]);
    }
  }
  if constexpr (K + 1 < 16) et_lu_step<K + 1>(v, r, st);
}

__device__ __forceinline__ float et_det16(const float (*R)[kRMax + 1], int r) {
  const int lane = threadIdx.x & 31;
  float v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = (lane < r && j < r) ? R[lane][j] : 0.f;
  EtLu st{1.f, 0, r >= 32 ? 0xffffffffu : ((1u << r) - 1u), false};
  et_lu_step<0>(v, r, st);
  if (st.zero) return 0.f;
  return st.parity ? -st.det : st.det;
}

struct EtShared {
  uint64_t* full;  // [2] move warps -> MLP warps: the batch's layer-0 rows are staged
  uint64_t* feat;  // [2] MLP warps -> move warps: the batch's final features are written
  uint64_t* dbar;  // [2] per MMA tile: the layer's MMAs have completed
  uint64_t* abar;  // [2] per MMA tile: the next layer's A operand is in TMEM
  int* abort;
};

__device__ __forceinline__ bool et_aborted(const EtShared& sh) { return *(volatile int*)sh.abort != 0; }
__device__ __forceinline__ void et_abort(const EtShared& sh, int* err) {
  if (atomicExch(sh.abort, 1) == 0) atomicExch(err, 1);
}

// The MMAs of site-wise layer l (1..L-1) for MMA tile mt: D = A W_l^T with A = hi + lo in TMEM,
// then a commit to the tile's mbarrier. One thread.
__device__ __forceinline__ void et_issue(uint32_t tmem, const float* wimg, int mt, int l, uint64_t* dbar) {
  const uint32_t d = tmem + mt * kEtTileCols, ah = d + kEtH, al = d + 2 * kEtH;
  const float* wl = wimg + (size_t)(l - 1) * 2 * kEtH * kEtH;
#pragma unroll
  for (int kk = 0; kk < kEtKT; ++kk) {
    const uint64_t bh = tc::smem_desc_kmajor(tc::smem_u32(wl + (size_t)(2 * kk) * kEtH * 8), 128, 256);
    const uint64_t bl = tc::smem_desc_kmajor(tc::smem_u32(wl + (size_t)(2 * kk + 1) * kEtH * 8), 128, 256);
    tc::mma_tf32_ta(d, ah + 8 * kk, bh, kEtIdesc, kk > 0 ? 1u : 0u);
    tc::mma_tf32_ta(d, al + 8 * kk, bh, kEtIdesc, 1u);
    tc::mma_tf32_ta(d, ah + 8 * kk, bl, kEtIdesc, 1u);
  }
  tc::mma_commit(dbar);
}

// MLP warps: the site-wise layers of the chunk's batches g0 .. g0 + nb - 1.
// Phase counters per MMA tile mt = 0, 1 (scalars, so that they stay in registers).
struct EtMlpState {
  uint32_t d0, d1;  // completed phases of dbar[mt] seen by this thread
  uint32_t a0, a1;  // completed phases of abar[mt] seen by the issuing thread
  uint32_t i0, i1;  // commits issued (issuing thread)
};

__device__ void et_mlp(const Net<float>& net, const EtShared& sh, int* err, const float* wimg, float* bbuf,
                       uint32_t tmem, int g0, int nb, EtMlpState& st) {
  constexpr int HC = kEtCols;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, col0 = (warp >> 2) * HC;
  const uint32_t lrow = (uint32_t)(32 * q) << 16;
  const bool issuer = threadIdx.x == 0;
  const int L = net.L;
  for (int tb = 0; tb < nb; ++tb) {
    if (et_aborted(sh)) return;
    const int gg = g0 + tb, buf = gg & 1;
    if (!tc::mbar_wait(&sh.full[buf], (uint32_t)(gg >> 1) & 1u, kEtPolls)) {
      et_abort(sh, err);
      return;
    }
    float* B = bbuf + (size_t)buf * kEtRows * kEtLd;
    // layer-1 input: the staged rows, split into the A halves of both tiles
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
      const float4* row = reinterpret_cast<const float4*>(B + (size_t)(mt * 128 + 32 * q + lane) * kEtLd + col0);
      float x[HC];
#pragma unroll
      for (int u = 0; u < HC / 4; ++u) {
        const float4 v = row[u];
        x[4 * u] = v.x;
        x[4 * u + 1] = v.y;
        x[4 * u + 2] = v.z;
        x[4 * u + 3] = v.w;
      }
      const uint32_t base = tmem + lrow + mt * kEtTileCols;
      et_store_split<HC>(base + kEtH + col0, base + 2 * kEtH + col0, x);
    }
    tc::tmem_wait_st();
    tc::fence_before_sync();
    tc::mbar_arrive(&sh.abar[0]);
    tc::mbar_arrive(&sh.abar[1]);
    if (issuer) {
      for (int mt = 0; mt < 2; ++mt) {
        if (!tc::mbar_wait(&sh.abar[mt], (mt ? st.a1 : st.a0) & 1u, kEtPolls)) {
          et_abort(sh, err);
          return;
        }
        if (mt) ++st.a1; else ++st.a0;
        tc::fence_after_sync();
        et_issue(tmem, wimg, mt, 1, &sh.dbar[mt]);
        if (mt) ++st.i1; else ++st.i0;
      }
    }
    for (int l = 1; l < L; ++l) {
      const float* bias = net.bias[l] + col0;
      const bool res = net.resid[l] != 0;
#pragma unroll 1
      for (int mt = 0; mt < 2; ++mt) {
        if (!tc::mbar_wait(&sh.dbar[mt], (mt ? st.d1 : st.d0) & 1u, kEtPolls)) {
          et_abort(sh, err);
          return;
        }
        if (mt) ++st.d1; else ++st.d0;
        tc::fence_after_sync();
        const uint32_t base = tmem + lrow + mt * kEtTileCols;
        float y[HC];
        {
          uint32_t d[HC / 8][8];
#pragma unroll
          for (int u = 0; u < HC / 8; ++u) tc::tmem_ld8_nowait(base + col0 + 8 * u, d[u]);
          tc::tmem_wait_ld();
#pragma unroll
          for (int u = 0; u < HC / 8; ++u)
#pragma unroll
            for (int j = 0; j < 8; ++j) y[8 * u + j] = __uint_as_float(d[u][j]) + __ldg(bias + 8 * u + j);
        }
        et_act<HC>(net.act, y);
        if (res) {  // the layer's input, hi + lo, read back from the A columns
#pragma unroll
          for (int u = 0; u < HC / 8; ++u) {
            uint32_t h[8], o[8];
            tc::tmem_ld8_nowait(base + kEtH + col0 + 8 * u, h);
            tc::tmem_ld8_nowait(base + 2 * kEtH + col0 + 8 * u, o);
            tc::tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 8; ++j) y[8 * u + j] += __uint_as_float(h[j]) + __uint_as_float(o[j]);
          }
        }
        if (l + 1 < L) {  // the next layer's A operand
          et_store_split<HC>(base + kEtH + col0, base + 2 * kEtH + col0, y);
          tc::tmem_wait_st();
          tc::fence_before_sync();
          tc::mbar_arrive(&sh.abar[mt]);
          if (issuer) {
            if (!tc::mbar_wait(&sh.abar[mt], (mt ? st.a1 : st.a0) & 1u, kEtPolls)) {
              et_abort(sh, err);
              return;
            }
            if (mt) ++st.a1; else ++st.a0;
            tc::fence_after_sync();
            et_issue(tmem, wimg, mt, l + 1, &sh.dbar[mt]);
            if (mt) ++st.i1; else ++st.i0;
          }
        } else {  // H'(L): the final features of the row
          float4* row = reinterpret_cast<float4*>(B + (size_t)(mt * 128 + 32 * q + lane) * kEtLd + col0);
#pragma unroll
          for (int u = 0; u < HC / 4; ++u) row[u] = make_float4(y[4 * u], y[4 * u + 1], y[4 * u + 2], y[4 * u + 3]);
        }
      }
    }
    tc::mbar_arrive(&sh.feat[buf]);
  }
}

// Move warp, staging: S and the layer-0 output rows of one move (lane = channel).
__device__ void et_stage(const LowrankArgs& a, const Net<float>& net, const int8_t* occ_s, const float* z0b,
                         uint32_t pm, float* rows, EtMeta& mt) {
  const int lane = threadIdx.x & 31, c = lane;
  const MoveDesc m = unpack_move(pm);
  const int kk = net.taps0, npairs = 2 * kk;  // (touched site, tap) pairs, one per lane
  int s_site = -1;
  if (lane < npairs) {
    const int t = lane < kk ? m.src : m.dst;
    int dx, dy;
    stencil_tap(net.stencil, a.k0, lane < kk ? lane : lane - kk, dx, dy);
    s_site = site_off(a.lat, t, -dx, -dy);
  }
  const unsigned act_mask = __ballot_sync(0xffffffffu, s_site >= 0);
  const unsigned same = __match_any_sync(0xffffffffu, s_site);
  const int first = __ffs(same & act_mask) - 1;
  const bool is_first = s_site >= 0 && first == lane;
  const unsigned firsts = __ballot_sync(0xffffffffu, is_first);
  const int nS = __popc(firsts);
  const int ps = s_site >= 0 ? __popc(firsts & ((1u << first) - 1u)) : -1;  // S index of pair `lane`
  const int n_src_old = occ_s[m.src] & 3, n_dst_old = occ_s[m.dst] & 3;
  const int n_src_new = move_new_state(m.kind, m.spin, true, n_src_old, n_dst_old);
  const int n_dst_new = move_new_state(m.kind, m.spin, false, n_src_old, n_dst_old);
  if (is_first) {
    const int n_old = occ_s[s_site] & 3;
    mt.site[ps] = (int16_t)s_site;
    mt.nold[ps] = (int8_t)n_old;
    mt.nnew[ps] = (int8_t)(s_site == m.src ? n_src_new : (s_site == m.dst ? n_dst_new : n_old));
  }
  if (lane == 0) mt.nS = nS;
  __syncwarp();
  // z0 of the sites of S
#pragma unroll 1
  for (int s0 = 0; s0 < nS; s0 += 6) {
    float z[6];
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      const int s = s0 + u;
      z[u] = s < nS ? __ldg(z0b + (size_t)mt.site[s] * kEtH + c) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 6; ++u)
      if (s0 + u < nS) rows[(s0 + u) * kEtLd + c] = z[u];
  }
  // layer-0 table deltas: pair p adds KE[t][n'_t][d] - KE[t][n_t][d] to the row of its site
  const int ts_src = net.per_site ? m.src : 0, ts_dst = net.per_site ? m.dst : 0;
#pragma unroll 1
  for (int p0 = 0; p0 < npairs; p0 += 9) {
    float dv[9];
    int dr[9];
#pragma unroll
    for (int u = 0; u < 9; ++u) {
      const int p = p0 + u;
      const int rp = __shfl_sync(0xffffffffu, ps, p & 31);
      dr[u] = p < npairs ? rp : -1;
      dv[u] = 0.f;
      if (dr[u] >= 0) {
        const bool fs = p < kk;
        const int d = fs ? p : p - kk;
        const int ts = fs ? ts_src : ts_dst, nn = fs ? n_src_new : n_dst_new, no = fs ? n_src_old : n_dst_old;
        dv[u] = __ldg(net.KE + (((size_t)ts * 4 + nn) * kk + d) * kEtH + c) -
                __ldg(net.KE + (((size_t)ts * 4 + no) * kk + d) * kEtH + c);
      }
    }
#pragma unroll
    for (int u = 0; u < 9; ++u)
      if (dr[u] >= 0) rows[dr[u] * kEtLd + c] += dv[u];
  }
  // residual embedding + activation
#pragma unroll 1
  for (int s0 = 0; s0 < nS; s0 += 6) {
    float z[6], e[6];
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      const int s = s0 + u;
      const bool on = s < nS;
      z[u] = on ? rows[s * kEtLd + c] : 0.f;
      e[u] = (on && net.resid[0])
                 ? __ldg(net.embed + ((size_t)(net.per_site ? mt.site[s] * 4 : 0) + mt.nnew[s]) * kEtH + c)
                 : 0.f;
    }
    et_act<6>(net.act, z);
#pragma unroll
    for (int u = 0; u < 6; ++u)
      if (s0 + u < nS) rows[(s0 + u) * kEtLd + c] = e[u] + z[u];
  }
}

// Move warp, after the site-wise layers: R of Eq. SMW and det R for one move. rows holds the
// final features H'(L) of the move's sites (overwritten with H'(L) - H(L)).
__device__ float et_finish(const LowrankArgs& a, const Net<float>& net, const int32_t* slot_s, const float* HLb,
                           const float* Binvb, const float* Ptb, uint32_t pm, float* rows, const EtMeta& mt,
                           EtScratch& sc) {
  const int lane = threadIdx.x & 31;
  const int N = a.lat.N, Ne = a.lat.Ne;
  const MoveDesc m = unpack_move(pm);
  const int nS = mt.nS;
  // electrons on S after the move: spin up first, then down, each in S order; rows and columns
  // of R follow the same list, so the order does not change det R
  int r = 0, r_up = 0;
  bool bad = false;
  for (int sp = 0; sp < 2; ++sp) {
    if (sp == 1) r_up = r;
    const int s = lane;  // nS <= kSMax < 32
    int slot = -1, mv = 0, site = 0;
    bool occ = false;
    if (s < nS) {
      site = mt.site[s];
      occ = (mt.nnew[s] >> sp) & 1;
      if (occ) {
        if ((mt.nold[s] >> sp) & 1) {
          slot = slot_s[sp * N + site];  // same electron, same orbital
        } else if (m.kind == 0) {
          slot = slot_s[sp * N + m.src];  // the hopping electron
          mv = 1;
        } else {
          slot = slot_s[sp * N + (site == m.src ? m.dst : m.src)];  // exchanged spin
          mv = 1;
        }
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, occ);
    if (occ) {
      const int pos = r + __popc(bal & ((1u << lane) - 1u));
      if (slot < 0) bad = true;
      if (pos < kRMax) {
        sc.slot[pos] = slot;
        sc.orb[pos] = sp * N + site;
        sc.sidx[pos] = s;
        sc.moved[pos] = mv;
      }
    }
    r += __popc(bal);
  }
  bad = __any_sync(0xffffffffu, bad);
  __syncwarp();
  if (r > kRMax || bad) return CUDART_NAN_F;
  // H'(L) - H(L) in place
#pragma unroll 1
  for (int s0 = 0; s0 < nS; s0 += 6) {
    float hl[6];
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      const int s = s0 + u;
      hl[u] = s < nS ? __ldg(HLb + (size_t)mt.site[s] * kEtH + lane) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 6; ++u)
      if (s0 + u < nS) rows[(s0 + u) * kEtLd + lane] -= hl[u];
  }
  __syncwarp();
  // electrons that kept their orbital: R[a][b] = delta_ab + (H'(L) - H(L))_{s_a} . Pt[s(a)][c_b],
  // one entry (a, b) per lane at a time
  const int rr = r * r;
  for (int q = lane; q < rr; q += 32) {
    const int aa = q / r, bb = q - aa * r;
    if (sc.moved[aa]) continue;
    const float4* x = reinterpret_cast<const float4*>(rows + sc.sidx[aa] * kEtLd);
    const float4* p = reinterpret_cast<const float4*>(Ptb + ((size_t)(aa >= r_up ? Ne : 0) + sc.slot[bb]) * kEtH);
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
    for (int u = 0; u < kEtH / 4; ++u) {
      const float4 xv = x[u], pv = __ldg(p + u);
      s0 = fmaf(xv.x, pv.x, s0);
      s1 = fmaf(xv.y, pv.y, s1);
      s2 = fmaf(xv.z, pv.z, s2);
      s3 = fmaf(xv.w, pv.w, s3);
    }
    sc.R[aa][bb] = (aa == bb ? 1.f : 0.f) + ((s0 + s1) + (s2 + s3));
  }
  // moved electrons: R[a][b] = (M0 + b)[o'_a] . Binv[c_b] + H'(L)_{s_a} . Pt[s(a)][c_b]; lanes over
  // the Ne entries of the first dot and the channels of the second, one warp sum per column
  for (int aa = 0; aa < r; ++aa) {
    if (!sc.moved[aa]) continue;
    const int s = sc.sidx[aa];
    const float xh = rows[s * kEtLd + lane] + __ldg(HLb + (size_t)mt.site[s] * kEtH + lane);
    const float* m0b = net.M0b + (size_t)sc.orb[aa] * Ne;
    const float* ptb = Ptb + (size_t)(aa >= r_up ? Ne : 0) * kEtH;
    constexpr int KK = 7;  // entries per lane per pass (224 per warp)
    for (int b0 = 0; b0 < r; b0 += 4) {
      float g[4];
      const float* br[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int sb = sc.slot[min(b0 + q, r - 1)];
        br[q] = Binvb + (size_t)sb * Ne;
        g[q] = xh * __ldg(ptb + (size_t)sb * kEtH + lane);
      }
      for (int k0 = 0; k0 < Ne; k0 += 32 * KK) {
        float v[KK], bv[4][KK];
#pragma unroll
        for (int u = 0; u < KK; ++u) {
          const int k = k0 + lane + 32 * u;
          const bool on = k < Ne;
          v[u] = on ? __ldg(m0b + k) : 0.f;
#pragma unroll
          for (int q = 0; q < 4; ++q) bv[q][u] = on ? __ldg(br[q] + k) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < KK; ++u)
#pragma unroll
          for (int q = 0; q < 4; ++q) g[q] = fmaf(v[u], bv[q][u], g[q]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) g[q] += __shfl_xor_sync(0xffffffffu, g[q], off);
        if (lane == b0 + q && b0 + q < r) sc.R[aa][lane] = g[q];
      }
    }
  }
  __syncwarp();
  return r <= 16 ? et_det16(sc.R, r) : warp_det_R<float>(sc.R, r);
}

// Move warps: stage batch tb and finish batch tb - 1 of the chunk, tb = 0 .. nb.
__device__ void et_work(const LowrankArgs& a, const Net<float>& net, const EtArgs& t, const EtShared& sh,
                        const int8_t* occ_s, const int32_t* slot_s, const float* z0b, const float* HLb,
                        const float* Binvb, const float* Ptb, const uint32_t* mlist, int nm, double* contrib,
                        float* bbuf, EtMeta* meta, EtScratch& sc, int g0, int nb) {
  const int w = (threadIdx.x >> 5) - kEtMlpWarps, lane = threadIdx.x & 31;
  for (int tb = 0; tb <= nb; ++tb) {
    if (et_aborted(sh)) return;
    if (tb < nb) {
      const int gg = g0 + tb, buf = gg & 1;
      float* B = bbuf + (size_t)buf * kEtRows * kEtLd;
      EtMeta* M = meta + buf * kEtMaxMoves;
      const int m0 = tb * t.mb, mc = min(t.mb, nm - m0);
      for (int j = w; j < mc; j += kEtWork) et_stage(a, net, occ_s, z0b, mlist[m0 + j], B + (size_t)j * t.rpm * kEtLd, M[j]);
      __syncwarp();
      if (!(t.inject && gg == 0)) tc::mbar_arrive(&sh.full[buf]);
    }
    if (tb >= 1) {
      const int gp = g0 + tb - 1, buf = gp & 1;
      if (!tc::mbar_wait(&sh.feat[buf], (uint32_t)(gp >> 1) & 1u, kEtPolls)) {
        et_abort(sh, t.err);
        return;
      }
      float* B = bbuf + (size_t)buf * kEtRows * kEtLd;
      const EtMeta* M = meta + buf * kEtMaxMoves;
      const int m0 = (tb - 1) * t.mb, mc = min(t.mb, nm - m0);
      for (int j = w; j < mc; j += kEtWork) {
        const uint32_t pm = mlist[m0 + j];
        const float det =
            et_finish(a, net, slot_s, HLb, Binvb, Ptb, pm, B + (size_t)j * t.rpm * kEtLd, M[j], sc);
        if (lane == 0) contrib[m0 + j] = move_coeff(a.lat, pm) * (double)det;
        __syncwarp();
      }
    }
  }
}

__global__ void __launch_bounds__(kEtThreads, 1) k_eloc_tc(LowrankArgs a, Net<float> net, EtArgs t) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  const int N = a.lat.N, Ne = a.lat.Ne;
  const EtLayout lay(t.nsw, N);
  float* wimg = reinterpret_cast<float*>(smem + lay.wimg);
  float* bbuf = reinterpret_cast<float*>(smem + lay.bbuf);
  EtMeta* meta = reinterpret_cast<EtMeta*>(smem + lay.meta);
  EtScratch* scr = reinterpret_cast<EtScratch*>(smem + lay.scr);
  uint32_t* mlist = reinterpret_cast<uint32_t*>(smem + lay.mlist);
  double* contrib = reinterpret_cast<double*>(smem + lay.contrib);
  int32_t* slot_s = reinterpret_cast<int32_t*>(smem + lay.slot);
  int8_t* occ_s = reinterpret_cast<int8_t*>(smem + lay.occ);
  __shared__ __align__(8) uint64_t bars[8];
  __shared__ uint32_t s_tmem;
  __shared__ int warp_cnt[kEtWarps];
  __shared__ double s_diag;
  __shared__ int s_abort;

  const int b = a.list ? a.list[blockIdx.x] : blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (a.status[b] & (SCALE_SAMPLE_BAD_COUNT | SCALE_SAMPLE_DOUBLE_OCC | SCALE_SAMPLE_SINGULAR)) {
    if (tid == 0) {
      a.out[b] = CUDART_NAN;
      if (a.move_count) a.move_count[b] = 0;
    }
    return;
  }
  for (int i = tid; i < N; i += kEtThreads) occ_s[i] = a.occ[(size_t)b * N + i];
  for (int o = tid; o < 2 * N; o += kEtThreads) slot_s[o] = a.slot_of_orb[(size_t)b * 2 * N + o];
  {
    const float4* src = reinterpret_cast<const float4*>(t.wimg);
    float4* dst = reinterpret_cast<float4*>(wimg);
    const int n4 = t.nsw * 2 * kEtH * kEtH / 4;
    for (int q = tid; q < n4; q += kEtThreads) dst[q] = __ldg(src + q);
    float4* bz = reinterpret_cast<float4*>(bbuf);
    for (int q = tid; q < 2 * kEtRows * kEtLd / 4; q += kEtThreads) bz[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  EtShared sh{bars, bars + 2, bars + 4, bars + 6, &s_abort};
  if (tid == 0) {
    for (int q = 0; q < 2; ++q) {
      tc::mbar_init(&sh.full[q], kEtWork * 32);
      tc::mbar_init(&sh.feat[q], kEtMlpWarps * 32);
      tc::mbar_init(&sh.dbar[q], 1);
      tc::mbar_init(&sh.abar[q], kEtMlpWarps * 32);
    }
    tc::mbar_fence_init();
    s_abort = 0;
  }
  if (warp == 0) tc::tmem_alloc(&s_tmem, kEtTmemCols);
  tc::fence_proxy_async();  // the weight tiles, written by generic stores, are read by the MMAs
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  if (tid == 0) s_diag = diag_energy(a, occ_s);

  const float* z0b = (const float*)a.z0 + (size_t)b * N * kEtH;
  const float* HLb = (const float*)a.HL + (size_t)b * N * kEtH;
  const float* Binvb = (const float*)a.Binv + (size_t)b * Ne * Ne;
  const float* Ptb = (const float*)a.Pt + (size_t)b * 2 * Ne * kEtH;
  EtMlpState st{0u, 0u, 0u, 0u, 0u, 0u};
  const int ncand = candidate_count(a);
  double total = 0.0;  // thread 0
  int nmoves = 0;
  int g = 0;  // batches so far (the phase of both buffers' mbarriers)
  for (int cs = 0; cs < ncand; cs += kMoveChunk) {
    const int ce = min(ncand, cs + kMoveChunk);
    const int nm = enumerate_chunk<kEtWarps>(a, occ_s, cs, ce, mlist, warp_cnt);
    const int nb = (nm + t.mb - 1) / t.mb;
    if (warp < kEtMlpWarps)
      et_mlp(net, sh, t.err, wimg, bbuf, tmem, g, nb, st);
    else
      et_work(a, net, t, sh, occ_s, slot_s, z0b, HLb, Binvb, Ptb, mlist, nm, contrib, bbuf, meta,
              scr[warp - kEtMlpWarps], g, nb);
    g += nb;
    __syncthreads();
    if (warp == 0) {  // fixed-order sum of the chunk
      double s = 0.0;
      for (int q = lane; q < nm; q += 32) s += contrib[q];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (lane == 0) {
        total += s;
        nmoves += nm;
      }
    }
    __syncthreads();
  }
  // after an early exit, MMAs may still be in flight: wait (bounded) for every commit
  if (tid == 0 && s_abort) {
    for (int mt = 0; mt < 2; ++mt)
      if ((mt ? st.i1 : st.i0) > (mt ? st.d1 : st.d0))
        tc::mbar_wait(&sh.dbar[mt], ((mt ? st.i1 : st.i0) - 1) & 1u, kEtPolls);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, kEtTmemCols);
  if (tid == 0) {
    a.out[b] = s_abort ? CUDART_NAN : s_diag + total;
    if (a.move_count) a.move_count[b] = nmoves;
  }
}

}  // namespace

// Largest affected set of any move of the lattice: the union of layer 0's stencil sites around
// the two ends of every NN / NNN bond (hops and t-J exchanges run on those bonds).
int et_rows_per_move(const scale_ctx* c, const std::vector<int32_t>& bonds) {
  const int kk = stencil_taps(c->arch.stencil, c->k0);
  int best = 0;
  for (size_t q = 0; q + 1 < bonds.size(); q += 2) {
    int sites[64];
    int n = 0;
    for (int e = 0; e < 2; ++e)
      for (int d = 0; d < kk; ++d) {
        int dx, dy;
        stencil_tap(c->arch.stencil, c->k0, d, dx, dy);
        const int s = site_off(c->lat, bonds[q + e], -dx, -dy);
        if (s < 0) continue;
        bool seen = false;
        for (int i = 0; i < n; ++i) seen = seen || sites[i] == s;
        if (!seen && n < 64) sites[n++] = s;
      }
    best = std::max(best, n);
  }
  return best;
}

size_t et_wimg_bytes(const scale_ctx* c) { return (size_t)(c->L - 1) * 2 * kEtH * kEtH * 4; }

// Shapes the batched kernel takes: mixed precision with TF32x3 site-wise layers, the SCALE
// layout, 32 channels, at least one site-wise layer, and a shared-memory plan that fits.
bool et_supported(const scale_ctx* c, int rows_per_move, int smem_optin) {
  if (c->fp64 || c->arch.precision != SCALE_PREC_MIXED || !c->lowrank_ok || c->h != kEtH || c->L < 2) return false;
  if (rows_per_move < 1 || rows_per_move > kSMax || 2 * stencil_taps(c->arch.stencil, c->k0) > 32) return false;
  const EtLayout lay(c->L - 1, c->N);
  return lay.total + 128 <= (size_t)smem_optin;
}

cudaError_t launch_build_et(scale_ctx* c) {
  if (!c->et_wimg) return cudaSuccess;
  const int total = (c->L - 1) * kEtKT * 2 * kEtH * 8;
  k_build_et_wimg<<<(total + 255) / 256, 256, 0, c->stream>>>(make_net<float>(c), c->L - 1, (float*)c->et_wimg);
  return cudaGetLastError();
}

// E_loc of the listed samples (list = nullptr: samples 0 .. n-1) by the batched kernel;
// cudaErrorNotSupported when the context's shape is not one it takes.
cudaError_t launch_eloc_tc(scale_ctx* c, double* eloc, const int32_t* list, int n) {
  if (!c->et_wimg) return cudaErrorNotSupported;
  if (n <= 0) return cudaSuccess;
  LowrankArgs a = make_args(c);
  a.out = eloc;
  a.move_count = c->move_count;
  a.list = list;
  EtArgs t{(const float*)c->et_wimg, c->L - 1, c->et_rows, std::min(kEtMaxMoves, kEtRows / c->et_rows), c->ace_err,
           c->et_inject};
  c->et_inject = 0;  // one-shot
  const EtLayout lay(t.nsw, c->N);
  const size_t smem = lay.total + 128;
  cudaError_t e = cudaFuncSetAttribute(k_eloc_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_eloc_tc<<<n, kEtThreads, smem, c->stream>>>(a, make_net<float>(c), t);
  return cudaGetLastError();
}

}  // namespace scale
