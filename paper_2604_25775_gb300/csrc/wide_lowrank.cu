// wide_lowrank.cu -- the cached update (Sec. II.C: Eq. neighbor, Eq. SMW) at the wide SCALE
// shapes of Table tab:model: one k x k conv with residual (3x3 box, or the 13-site plus of
// SCALE-L), then site-wise layers up to the last width h_L (SCALE-L: 384, then 4 x 512;
// SCALE-XL: 640, then 4 x 1280). At these widths the rows of a move do not fit the per-warp
// shared memory of the narrow kernel, so the affected rows of many moves are gathered into
// one buffer and the site-wise layers run on it as row GEMMs (tcgen05 at the Table widths),
// between a staging kernel and a finishing kernel that each take one warp per move:
//   1. enumeration: the allowed moves of every sample in the order of the narrow path,
//      packed by a device-side scan (no host synchronisation);
//   2. per chunk of moves, staging: the affected sites S of the move and the layer-0 rows
//        x_s = E_s[n'_s] + act(z0_s + sum over (t, d) of KE[t][n'_t][d] - KE[t][n_t][d]),
//      one row slot per site of S (wl_rows slots per move);
//   3. the site-wise layers 1 .. L-1 on every row of the chunk (the network's own kernels);
//   4. finishing: the electrons on S after the move and R of Eq. SMW,
//        R[a][b] = delta_ab + (H'(L) - H(L))_{s_a} . Pt[s(a)][c_b]              (orbital kept)
//                = (M0 + proj_b)[o'_a] . Binv[c_b] + H'(L)_{s_a} . Pt[s(a)][c_b]  (moved)
//      det R by LU with partial pivoting, and the move's term coeff * det R;
//   5. E_loc = diagonal + the terms in enumeration order, in FP64.
// scale_load builds the cache: z0 from the layer-0 table, H(L) from the load's forward, the
// FP64 inverse and Pt = W Phi^-1. Commits are not offered at these shapes.
#include <algorithm>
#include <set>

#include "eloc_common.cuh"

namespace scale {

namespace {

// One move of a chunk, written by its staging warp and read by its finishing warp.
struct WlMeta {
  int b;        // sample; -1 for a chunk slot past the last move
  uint32_t pm;  // packed move (eloc_common.cuh)
  int nS;
  int16_t site[kSMax];
  int8_t nold[kSMax], nnew[kSMax];
};

template <typename T>
struct WideView {
  Lattice lat;
  int h, hl, k0, taps0, stencil, per_site, res0, act, rpm;
  const int8_t* occ;
  const int32_t* slot_of_orb;
  const int32_t* status;
  const T* embed;  // [Ns][4][h]
  const T* bias0;  // [h]
  const T* KE;     // [Ns][4][taps0][h]
  const T* z0;     // [B][N][h]
  const T* HL;     // [B][N][hl]
  const T* Binv;   // [B][Ne][Ne]
  const T* Pt;     // [B][2][Ne][hl]
  const T* M0b;    // [2N][Ne]
  const uint32_t* moves;  // packed moves of all samples, [total]
  const int32_t* owner;   // sample of each packed move
  const int64_t* off;     // [B+1] offsets of each sample's moves
  int B;
  WlMeta* meta;           // [chunk]
};

template <typename T>
__device__ __forceinline__ T act_wide(int act, T z) {
  if constexpr (sizeof(T) == 4) return act_fast(act, z);  // the tensor-core layers' activation
  else return act_fn<T>(act, z);
}

// M0b[o][k] = M0[o][k] + proj_b[s(o) Ne + k]
template <typename T>
__global__ void k_wide_m0b(const T* __restrict__ M0, const T* __restrict__ pb, int N, int Ne, T* __restrict__ out) {
  const size_t total = (size_t)2 * N * Ne;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const size_t o = q / Ne, k = q - o * Ne;
    out[q] = M0[q] + pb[(o / N) * Ne + k];
  }
}

// z0[b][i][c] = bias0[c] + sum over the taps d of KE[t][n_t][d][c], t = i + offset(d): the
// layer-0 pre-activation of the loaded samples from the layer-0 table.
template <typename T>
__global__ void k_wide_z0(WideView<T> v, int B, T* __restrict__ z0) {
  const int N = v.lat.N, h = v.h, kk = v.taps0;
  const size_t total = (size_t)B * N * h;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(q % h);
    const size_t bi = q / h;
    const int i = (int)(bi % N);
    const int b = (int)(bi / N);
    T acc = v.bias0[c];
    for (int d = 0; d < kk; ++d) {
      int dx, dy;
      stencil_tap(v.stencil, v.k0, d, dx, dy);
      const int t = site_off(v.lat, i, dx, dy);
      if (t < 0) continue;
      const int n = v.occ[(size_t)b * N + t] & 3;
      acc += v.KE[(((size_t)(v.per_site ? t : 0) * 4 + n) * kk + d) * h + c];
    }
    z0[q] = acc;
  }
}

// Pt[b][s][c][j] = sum_k Binv[b][c][k] proj_w[j][s Ne + k]: a GEMM per (sample, spin), CTA
// tiles of 64 x 64 outputs, 4 x 4 per thread, K staged 32 at a time through shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_wide_project(int Ne, int hl, int b0, const T* __restrict__ Binv,
                                                      const T* __restrict__ proj_w, T* __restrict__ Pt) {
  __shared__ T As[32][65];  // As[k][c]
  __shared__ T Ws[32][65];  // Ws[k][j]
  const int b = b0 + (int)(blockIdx.z >> 1), s = blockIdx.z & 1;
  const int c0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
  const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
  const T* Bb = Binv + (size_t)b * Ne * Ne;
  T acc[4][4] = {};
  for (int k0 = 0; k0 < Ne; k0 += 32) {
    for (int q = tid; q < 64 * 32; q += 256) {
      const int rr = q >> 5, kk = q & 31;  // Binv row c0 + rr, k0 + kk: consecutive threads along k
      const int c = c0 + rr, k = k0 + kk;
      As[kk][rr] = (c < Ne && k < Ne) ? Bb[(size_t)c * Ne + k] : T(0);
      const int j = j0 + rr;
      Ws[kk][rr] = (j < hl && k < Ne) ? proj_w[(size_t)j * 2 * Ne + s * Ne + k] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 32; ++kk) {
      T a[4], w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[kk][tr + 16 * u];
        w[u] = Ws[kk][tc + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * w[v];
    }
    __syncthreads();
  }
  T* out = Pt + ((size_t)b * 2 + s) * Ne * hl;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int c = c0 + tr + 16 * u;
    if (c >= Ne) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = j0 + tc + 16 * v;
      if (j < hl) out[(size_t)c * hl + j] = acc[u][v];
    }
  }
}

// The allowed moves of every sample in enumeration order. Counting pass (off == nullptr):
// count[b] and the diagonal energy; packing pass: the moves at off[b] with their owner.
template <int NW>
__global__ void __launch_bounds__(32 * NW) k_wl_enum(LowrankArgs a, const int64_t* __restrict__ off,
                                                     uint32_t* __restrict__ moves, int32_t* __restrict__ owner,
                                                     int32_t* __restrict__ count, double* __restrict__ diag) {
  extern __shared__ unsigned char smem_raw[];
  uint32_t* mlist = reinterpret_cast<uint32_t*>(smem_raw);           // [kMoveChunk]
  int8_t* occ_s = reinterpret_cast<int8_t*>(mlist + kMoveChunk);      // [N]
  __shared__ int warp_cnt[NW];
  const int b = blockIdx.x, N = a.lat.N, tid = threadIdx.x;
  for (int i = tid; i < N; i += blockDim.x) occ_s[i] = a.occ[(size_t)b * N + i];
  __syncthreads();
  const int total = candidate_count(a);
  int nm = 0;
  for (int cs = 0; cs < total; cs += kMoveChunk) {
    const int n = enumerate_chunk<NW>(a, occ_s, cs, min(total, cs + kMoveChunk), mlist, warp_cnt);
    if (off)
      for (int q = tid; q < n; q += blockDim.x) {
        moves[off[b] + nm + q] = mlist[q];
        owner[off[b] + nm + q] = b;
      }
    nm += n;
    __syncthreads();
  }
  if (!off && tid == 0) {
    count[b] = nm;
    diag[b] = diag_energy(a, occ_s);
  }
}

constexpr int kWlWarps = 4;  // warps (moves) per CTA of the staging and finishing kernels

// Staging: warp j of the chunk takes move g0 + j. SPLIT: rows as TF32 (hi, lo) halves.
template <typename T, bool SPLIT>
__global__ void __launch_bounds__(32 * kWlWarps) k_wl_stage(WideView<T> v, int64_t g0, int MC, T* __restrict__ rows,
                                                            T* __restrict__ rows_lo, int32_t* __restrict__ nvalid) {
  __shared__ T buf[kWlWarps][kSMax][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * kWlWarps + warp;
  if (j >= MC) return;  // whole warp
  const int64_t total = v.off[v.B];
  if (j == 0 && lane == 0) *nvalid = (int32_t)max((int64_t)0, min((int64_t)MC, total - g0));
  WlMeta& m = v.meta[j];
  const int64_t g = g0 + j;
  if (g >= total) {
    if (lane == 0) m.b = -1;
    return;
  }
  const int b = v.owner[g];
  const uint32_t pm = v.moves[g];
  const MoveDesc mv = unpack_move(pm);
  const int N = v.lat.N, h = v.h, kk = v.taps0, npairs = 2 * kk;
  const int8_t* ob = v.occ + (size_t)b * N;
  // pairs (touched site t, tap d), one per lane: the site reached is t - offset(d)
  int s_site = -1;
  if (lane < npairs) {
    const int t = lane < kk ? mv.src : mv.dst;
    int dx, dy;
    stencil_tap(v.stencil, v.k0, lane % kk, dx, dy);
    s_site = site_off(v.lat, t, -dx, -dy);
  }
  const unsigned act_mask = __ballot_sync(0xffffffffu, s_site >= 0);
  const unsigned same = __match_any_sync(0xffffffffu, s_site);
  const int first = __ffs(same & act_mask) - 1;
  const bool is_first = s_site >= 0 && first == lane;
  const unsigned firsts = __ballot_sync(0xffffffffu, is_first);
  const int n_src_old = ob[mv.src] & 3, n_dst_old = ob[mv.dst] & 3;
  const int n_src_new = move_new_state(mv.kind, mv.spin, true, n_src_old, n_dst_old);
  const int n_dst_new = move_new_state(mv.kind, mv.spin, false, n_src_old, n_dst_old);
  int pair_s = -1;  // index in S of this lane's pair
  if (s_site >= 0) {
    pair_s = __popc(firsts & ((1u << first) - 1u));
    if (is_first) {
      const int n_old = ob[s_site] & 3;
      m.site[pair_s] = (int16_t)s_site;
      m.nold[pair_s] = (int8_t)n_old;
      m.nnew[pair_s] = (int8_t)(s_site == mv.src ? n_src_new : (s_site == mv.dst ? n_dst_new : n_old));
    }
  }
  const int nS = __popc(firsts);
  if (lane == 0) {
    m.b = b;
    m.pm = pm;
    m.nS = nS;
  }
  __syncwarp();
  const int ts_src = v.per_site ? mv.src : 0, ts_dst = v.per_site ? mv.dst : 0;
  const T* z0b = v.z0 + (size_t)b * N * h;
  const size_t row0 = (size_t)j * v.rpm;
  for (int c0 = 0; c0 < h; c0 += 32) {
    const int c = c0 + lane;
    const bool on = c < h;
    for (int s = 0; s < nS; ++s) buf[warp][s][lane] = on ? z0b[(size_t)m.site[s] * h + c] : T(0);
    __syncwarp();
    for (int p = 0; p < npairs; ++p) {
      const int ps = __shfl_sync(0xffffffffu, pair_s, p);
      if (ps >= 0 && on) {
        const bool fs = p < kk;
        const int d = fs ? p : p - kk;
        const int ts = fs ? ts_src : ts_dst, nn = fs ? n_src_new : n_dst_new, no = fs ? n_src_old : n_dst_old;
        buf[warp][ps][lane] +=
            v.KE[(((size_t)ts * 4 + nn) * kk + d) * h + c] - v.KE[(((size_t)ts * 4 + no) * kk + d) * h + c];
      }
    }
    __syncwarp();
    if (on) {
      for (int s = 0; s < v.rpm; ++s) {
        T x = T(0);  // padding slots past S hold zeros
        if (s < nS) {
          const int site = m.site[s];
          x = act_wide<T>(v.act, buf[warp][s][lane]);
          if (v.res0) x += v.embed[((size_t)(v.per_site ? site : 0) * 4 + m.nnew[s]) * h + c];
        }
        const size_t q = (row0 + s) * h + c;
        if constexpr (SPLIT) {
          uint32_t hi, lo;
          split_tf32((float)x, hi, lo);
          rows[q] = __uint_as_float(hi);
          rows_lo[q] = __uint_as_float(lo);
        } else {
          rows[q] = x;
        }
      }
    }
    __syncwarp();
  }
}

// Finishing: R of Eq. SMW from the new features on S, det R, the move's term.
template <typename T>
__global__ void __launch_bounds__(32 * kWlWarps) k_wl_finish(WideView<T> v, int64_t g0, int MC,
                                                             const T* __restrict__ feat, double* __restrict__ terms) {
  extern __shared__ __align__(16) unsigned char wsm[];  // [kWlWarps][hl]: the row a's vector
  __shared__ T Rs[kWlWarps][kRMax][kRMax + 1];
  __shared__ int sl_slot[kWlWarps][kRMax], sl_sidx[kWlWarps][kRMax], sl_moved[kWlWarps][kRMax], sl_orb[kWlWarps][kRMax];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * kWlWarps + warp;
  if (j >= MC) return;  // whole warp
  const WlMeta& m = v.meta[j];
  const int b = m.b;
  if (b < 0) return;
  const int64_t g = g0 + j;
  const MoveDesc mv = unpack_move(m.pm);
  const int N = v.lat.N, Ne = v.lat.Ne, hl = v.hl, nS = m.nS;
  const int32_t* so = v.slot_of_orb + (size_t)b * 2 * N;
  T(*R)[kRMax + 1] = Rs[warp];
  int* slot = sl_slot[warp];
  int* sidx = sl_sidx[warp];
  int* moved = sl_moved[warp];
  int* orb = sl_orb[warp];
  // electrons on S after the move: spin up first, then down, each in S order
  int r = 0, r_up = 0;
  bool bad = false;
  for (int sp = 0; sp < 2; ++sp) {
    if (sp == 1) r_up = r;
    const int s = lane;
    int sl = -1, mvd = 0;
    bool occ = false;
    if (s < nS) {
      occ = (m.nnew[s] >> sp) & 1;
      if (occ) {
        const int site = m.site[s];
        if ((m.nold[s] >> sp) & 1) {
          sl = so[sp * N + site];
        } else if (mv.kind == 0) {
          sl = so[sp * N + mv.src];
          mvd = 1;
        } else {
          sl = so[sp * N + (site == mv.src ? mv.dst : mv.src)];
          mvd = 1;
        }
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, occ);
    if (occ) {
      const int pos = r + __popc(bal & ((1u << lane) - 1u));
      if (sl < 0) bad = true;
      if (pos < kRMax) {
        slot[pos] = sl;
        sidx[pos] = s;
        moved[pos] = mvd;
        orb[pos] = sp * N + m.site[s];
      }
    }
    r += __popc(bal);
  }
  bad = __any_sync(0xffffffffu, bad);
  __syncwarp();
  if (r > kRMax || bad) {
    if (lane == 0) terms[g] = CUDART_NAN;
    return;
  }
  // R, one row a at a time: its feature row (H'(L) - H(L) if the orbital is kept) staged in
  // shared memory once, then dotted against the Pt rows of its spin four columns per pass
  // (lanes over channels, one reduction round per pass)
  const T* Ptb = v.Pt + (size_t)b * 2 * Ne * hl;
  const T* HLb = v.HL + (size_t)b * N * hl;
  const T* Bb = v.Binv + (size_t)b * Ne * Ne;
  T* dh = reinterpret_cast<T*>(wsm) + (size_t)warp * hl;
  for (int a = 0; a < r; ++a) {
    const int sp = a >= r_up;
    const int s = sidx[a];
    const bool kept = !moved[a];
    const T* x = feat + ((size_t)j * v.rpm + s) * hl;
    const T* hrow = HLb + (size_t)m.site[s] * hl;
    for (int c = lane; c < hl; c += 32) dh[c] = kept ? x[c] - hrow[c] : x[c];
    __syncwarp();
    for (int b0 = 0; b0 < r; b0 += 4) {
      const T* p[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) p[u] = Ptb + ((size_t)sp * Ne + slot[min(b0 + u, r - 1)]) * hl;
      T acc[4] = {T(0), T(0), T(0), T(0)};
      for (int c = lane; c < hl; c += 32) {
        const T d = dh[c];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] += d * p[u][c];
      }
      if (!kept) {  // + (M0 + proj_b)[o'_a] . Binv[c_b]
        const T* mb = v.M0b + (size_t)orb[a] * Ne;
        for (int k = lane; k < Ne; k += 32) {
          const T mk = mb[k];
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[u] += mk * Bb[(size_t)slot[min(b0 + u, r - 1)] * Ne + k];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
      if (lane == 0)
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (b0 + u < r) R[a][b0 + u] = (kept && a == b0 + u ? T(1) : T(0)) + acc[u];
    }
    __syncwarp();
  }
  __syncwarp();
  const T det = warp_det_R<T>(R, r);
  if (lane == 0) terms[g] = move_coeff(v.lat, m.pm) * (double)det;
}

// E_loc = diagonal + the terms of the sample's moves in enumeration order.
__global__ void k_wl_reduce(int B, const int64_t* __restrict__ off, const double* __restrict__ diag,
                            const double* __restrict__ terms, const int32_t* __restrict__ status,
                            double* __restrict__ eloc) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  if (status[b] & (SCALE_SAMPLE_BAD_COUNT | SCALE_SAMPLE_DOUBLE_OCC | SCALE_SAMPLE_SINGULAR)) {
    eloc[b] = CUDART_NAN;
    return;
  }
  double e = diag[b];
  for (int64_t g = off[b]; g < off[b + 1]; ++g) e += terms[g];
  eloc[b] = e;
}

template <typename T>
WideView<T> make_view(scale_ctx* c) {
  WideView<T> v{};
  const scale_arch& a = c->arch;
  v.lat = c->lat;
  v.h = c->h;
  v.hl = ace_width_out(a, c->L - 1);
  v.k0 = c->k0;
  v.taps0 = stencil_taps(a.stencil, c->k0);
  v.stencil = a.stencil;
  v.per_site = a.per_site_embed;
  v.res0 = a.residual[0];
  v.act = a.act;
  v.rpm = c->wl_rows;
  v.occ = c->occ;
  v.slot_of_orb = c->slot_of_orb;
  v.status = c->status;
  const T* base = c->fp64 ? (const T*)c->params64 : (const T*)c->params32;
  v.embed = base;
  const int64_t ne = (int64_t)(a.per_site_embed ? c->N : 1) * 4 * c->h;
  v.bias0 = base + ne + (int64_t)v.taps0 * c->h * c->h;  // layer 0: kernel [taps][h][h], then bias
  v.KE = (const T*)c->KE;
  v.z0 = (const T*)c->z0;
  v.HL = (const T*)c->HL;
  v.Binv = (const T*)c->Binv;
  v.Pt = (const T*)c->Pt;
  v.M0b = (const T*)c->M0b;
  const size_t cap = std::max(1, c->max_moves);
  v.moves = (const uint32_t*)c->full_moves;
  v.owner = c->full_moves + (size_t)c->B_max * cap;
  v.off = c->full_offsets;
  v.B = c->B;
  v.meta = (WlMeta*)c->wl_meta;
  return v;
}

// Offset of proj_w in the flat parameters of the wide SCALE layout (embed; per layer kernel
// and bias; proj_w; proj_b).
int64_t proj_w_offset(const scale_ctx* c) {
  const scale_arch& a = c->arch;
  int64_t p = (int64_t)(a.per_site_embed ? c->N : 1) * 4 * c->h;
  for (int l = 0; l < c->L; ++l)
    p += (int64_t)stencil_taps(a.stencil, a.ksize[l]) * ace_width_in(a, l) * ace_width_out(a, l) +
         ace_width_out(a, l);
  return p;
}

template <typename T>
cudaError_t wide_cache_t(scale_ctx* c, int B) {
  const WideView<T> v = make_view<T>(c);
  const size_t total = (size_t)B * c->N * c->h;
  k_wide_z0<T><<<(unsigned)std::min<size_t>((total + 255) / 256, 152 * 32), 256, 0, c->stream>>>(v, B, (T*)c->z0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const T* base = c->fp64 ? (const T*)c->params64 : (const T*)c->params32;
  for (int b0 = 0; b0 < B; b0 += 32768) {  // grid z: two spins per sample, at most 65535
    const dim3 grid((c->Ne + 63) / 64, (v.hl + 63) / 64, 2 * std::min(32768, B - b0));
    k_wide_project<T><<<grid, 256, 0, c->stream>>>(c->Ne, v.hl, b0, (const T*)c->Binv, base + proj_w_offset(c),
                                                   (T*)c->Pt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t wide_eloc_t(scale_ctx* c, double* eloc) {
  WideView<T> v = make_view<T>(c);
  const LowrankArgs a = make_args(c);
  const int B = c->B, N = c->N;
  const size_t cap = std::max(1, c->max_moves);
  uint32_t* moves = (uint32_t*)c->full_moves;
  int32_t* owner = c->full_moves + (size_t)c->B_max * cap;
  const size_t esm = kMoveChunk * 4 + N;
  k_wl_enum<4><<<B, 128, esm, c->stream>>>(a, nullptr, moves, owner, c->move_count, c->full_diag);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = launch_offsets(c, B, c->move_count, 0, c->full_offsets)) != cudaSuccess) return e;
  k_wl_enum<4><<<B, 128, esm, c->stream>>>(a, c->full_offsets, moves, owner, c->move_count, c->full_diag);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // a stand-in lattice of wl_rows sites in a line: row slot s of move j is "site" s of
  // "configuration" j, which the site-wise layers read as row j * wl_rows + s
  Lattice rl{};
  rl.Lx = c->wl_rows;
  rl.Ly = 1;
  rl.pbc_x = rl.pbc_y = 1;
  rl.N = c->wl_rows;
  const int MC = c->wl_chunk;
  const int h = c->h;
  const long long rows = (long long)MC * c->wl_rows;
  const bool split = !c->fp64 && ace_tc_layer(c, 1);
  const int64_t bound = (int64_t)B * (int64_t)cap;  // the device-side total is at most this
  T* ra = (T*)c->act_a;
  const size_t fsm = (size_t)kWlWarps * v.hl * sizeof(T);  // the finishing warps' row vectors
  if (fsm > 48 * 1024 &&
      (e = cudaFuncSetAttribute(k_wl_finish<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm)) != cudaSuccess)
    return e;
  for (int64_t g0 = 0; g0 < bound; g0 += MC) {
    const unsigned grid = (unsigned)((MC + kWlWarps - 1) / kWlWarps);
    if (split)
      k_wl_stage<T, true><<<grid, 32 * kWlWarps, 0, c->stream>>>(v, g0, MC, ra, ra + rows * h, c->full_vcount);
    else
      k_wl_stage<T, false><<<grid, 32 * kWlWarps, 0, c->stream>>>(v, g0, MC, ra, nullptr, c->full_vcount);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    void* out = nullptr;
    if ((e = launch_ace_layers(c, rl, 1, c->L, c->act_a, c->act_b, rows, split, c->full_vcount, &out)) != cudaSuccess)
      return e;
    k_wl_finish<T><<<grid, 32 * kWlWarps, fsm, c->stream>>>(v, g0, MC, (const T*)out, c->full_coeff);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_wl_reduce<<<(B + 127) / 128, 128, 0, c->stream>>>(B, c->full_offsets, c->full_diag, c->full_coeff, c->status,
                                                       eloc);
  return cudaGetLastError();
}

}  // namespace

// One residual (or plain) conv of the 3x3 box or the 13-site plus as layer 0, site-wise layers
// after it: the layouts whose (touched site, tap) pairs fit one warp.
bool wide_lowrank_shapes(const scale_arch& a) {
  if (a.family != SCALE_FAMILY_WIDE || a.n_conv != 1) return false;
  const bool box = a.stencil == SCALE_STENCIL_BOX && (a.ksize[0] == 1 || a.ksize[0] == 3);
  const bool plus = a.stencil == SCALE_STENCIL_DISK && (a.ksize[0] == 3 || a.ksize[0] == 5);
  if (!box && !plus) return false;
  for (int l = 1; l < a.n_layers; ++l)
    if (a.ksize[l] != 1) return false;
  return true;
}

// Largest affected set of a move: the union of layer 0's stencil around the two touched sites
// of a bond (NN, NNN when t' != 0), as offsets (wrapping on a small lattice can only merge
// sites).
int wide_rows_per_move(const scale_system& s, const scale_arch& a) {
  const int k = a.ksize[0], r = (k - 1) / 2;
  std::vector<std::pair<int, int>> offs;
  for (int dy = -r; dy <= r; ++dy)
    for (int dx = -r; dx <= r; ++dx)
      if (a.stencil == SCALE_STENCIL_BOX || dx * dx + dy * dy <= r * r) offs.push_back({dx, dy});
  std::vector<std::pair<int, int>> bonds = {{1, 0}, {0, 1}};
  if (s.tp != 0.0) {
    bonds.push_back({1, 1});
    bonds.push_back({1, -1});
  }
  int best = 1;
  for (const auto& bd : bonds) {
    std::set<std::pair<int, int>> u;
    for (const auto& o : offs) {
      u.insert(o);
      u.insert({o.first + bd.first, o.second + bd.second});
    }
    best = std::max(best, (int)u.size());
  }
  return std::min(best, kSMax);
}

size_t wide_meta_bytes() { return sizeof(WlMeta); }

cudaError_t launch_wide_params(scale_ctx* c) {
  // the layer-0 table KE[t][n][d] = K0[d]^T E_t[n] (layer 0 has the narrow layout: h -> h)
  cudaError_t e = launch_build_ke(c);
  if (e != cudaSuccess) return e;
  // M0b = M0 + proj_b[s(o)]
  const int64_t pb = proj_w_offset(c) + (int64_t)ace_width_out(c->arch, c->L - 1) * 2 * c->Ne;
  if (c->fp64) {
    k_wide_m0b<double><<<512, 256, 0, c->stream>>>((const double*)c->M0_64, c->params64 + pb, c->N, c->Ne,
                                                  (double*)c->M0b);
  } else {
    k_wide_m0b<float><<<512, 256, 0, c->stream>>>(c->M0_32, c->params32 + pb, c->N, c->Ne, (float*)c->M0b);
  }
  return cudaGetLastError();
}

cudaError_t launch_wide_cache(scale_ctx* c, int B) {
  return c->fp64 ? wide_cache_t<double>(c, B) : wide_cache_t<float>(c, B);
}

cudaError_t launch_wide_eloc(scale_ctx* c, double* eloc) {
  return c->fp64 ? wide_eloc_t<double>(c, eloc) : wide_eloc_t<float>(c, eloc);
}

}  // namespace scale
