// move.cuh -- one connected configuration n -> n' handled by one warp (Sec. II.C).
//
//   1. touched sites T = {src, dst} ("exchange" set of Sec. II.C);
//   2. affected sites S = union over t in T of the layer-0 stencil around t (Eq. neighbor);
//      the later layers are site-wise, so S does not grow;
//   3. new features on S: layer-0 pre-activation z0' = z0 + sum over (t, d) of
//      KE[t][n'_t][d] - KE[t][n_t][d], then the residual / activation and the site-wise
//      layers; Delta H = H'(L) - H(L);
//   4. the electrons on S after the move, each with its determinant row (slot) c_a and new
//      orbital o'_a; the rank-r matrix of Eq. SMW with U = the changed rows,
//        R[a][b] = M'[o'_a] . Binv[c_b]
//                = [a moved ? G(o'_a, c_b) : delta_ab] + Delta H_{s_a} . Pt[s_a][c_b],
//        G(o, c) = (M0[o] + proj_b[s]) . Binv[c] + H(L)_i . Pt[s][c],
//      is A = I_r + V^T Phi^-1 U with V^T = Phi'_C - Phi_C;
//   5. det R by LU with partial pivoting (lane j owns column j).
// det R is the slot-order ratio det Phi'/det Phi; the moved electrons keep their rows.
#pragma once

#include "scale_internal.cuh"

namespace scale {

constexpr int kSMax = 18;   // affected sites for two touched sites and a 3x3 stencil
constexpr int kRMax = 32;   // electrons on the affected sites (lane per column)

template <typename T>
struct MoveScratch {
  int nS, r, kind, src, dst, spin;
  int site[kSMax];
  int nold[kSMax], nnew[kSMax];
  int pair_s[2 * 9];         // S index of each (touched site, offset) pair, -1 if none
  int slot[kRMax], orb[kRMax], sidx[kRMax], moved[kRMax];
  T feat[kSMax][kMaxH];      // working features, Delta H at the end
  T R[kRMax][kRMax + 1];
};

// Per-sample views used by the move routines.
template <typename T>
struct SampleView {
  const int8_t* occ;          // [N] (shared memory copy)
  const int32_t* slot_of_orb; // [2N]
  const T* z0;                // [N][h]
  const T* HL;                // [N][h]
  const T* Binv;              // [Ne][Ne]
  const T* Pt;                // [2][Ne][h]
};

__device__ __forceinline__ int move_new_state(int kind, int spin, bool is_src, int n_src, int n_dst) {
  if (kind == 0) return is_src ? (n_src & ~(1 << spin)) : (n_dst | (1 << spin));
  return is_src ? n_dst : n_src;  // exchange swaps the two sites' states
}

// Validity of a move against the current occupations (the model's space).
__device__ __forceinline__ bool move_allowed(const Lattice& lat, int kind, int src, int dst, int spin,
                                             const int8_t* occ) {
  if (kind < 0 || src == dst || src < 0 || dst < 0 || src >= lat.N || dst >= lat.N) return false;
  const int a = occ[src], b = occ[dst];
  if (kind == 0) {
    if (spin < 0 || spin > 1) return false;
    if (!((a >> spin) & 1) || ((b >> spin) & 1)) return false;
    if (lat.model == SCALE_MODEL_TJ && b != 0) return false;
    return true;
  }
  // exchange: opposite single spins
  return (a == 1 && b == 2) || (a == 2 && b == 1);
}

// Steps 1-3: S, new features and Delta H in ms.feat. All lanes of the warp participate.
template <typename T>
__device__ void move_features(const Lattice& lat, const Net<T>& net, int k0, const SampleView<T>& sv,
                              MoveScratch<T>& ms, T (*z0_new)[kMaxH] = nullptr) {
  const int lane = threadIdx.x & 31;
  const int h = net.h, r0 = (k0 - 1) / 2, kk = k0 * k0;
  const int npairs = 2 * kk;
  // pairs (t, d): t = src (pair < kk) or dst; the site reached is t - d
  int s_site = -1;
  if (lane < npairs) {
    const int t = (lane < kk) ? ms.src : ms.dst;
    const int d = lane % kk;
    const int dx = d % k0 - r0, dy = d / k0 - r0;
    s_site = site_off(lat, t, -dx, -dy);
  }
  const unsigned act_mask = __ballot_sync(0xffffffffu, s_site >= 0);
  const unsigned same = __match_any_sync(0xffffffffu, s_site);
  const int first = __ffs(same & act_mask) - 1;
  const bool is_first = (s_site >= 0) && (first == lane);
  const unsigned firsts = __ballot_sync(0xffffffffu, is_first);
  if (s_site >= 0) {
    const int pos = __popc(firsts & ((1u << first) - 1u));
    ms.pair_s[lane] = pos;
    if (is_first) {
      ms.site[pos] = s_site;
      const int n_old = sv.occ[s_site] & 3;
      int n_new = n_old;
      if (s_site == ms.src) n_new = move_new_state(ms.kind, ms.spin, true, sv.occ[ms.src], sv.occ[ms.dst]);
      if (s_site == ms.dst) n_new = move_new_state(ms.kind, ms.spin, false, sv.occ[ms.src], sv.occ[ms.dst]);
      ms.nold[pos] = n_old;
      ms.nnew[pos] = n_new;
    }
  } else if (lane < npairs) {
    ms.pair_s[lane] = -1;
  }
  if (lane == 0) ms.nS = __popc(firsts);
  __syncwarp();
  const int nS = ms.nS;
  const int n_src_old = sv.occ[ms.src] & 3, n_dst_old = sv.occ[ms.dst] & 3;
  const int n_src_new = move_new_state(ms.kind, ms.spin, true, n_src_old, n_dst_old);
  const int n_dst_new = move_new_state(ms.kind, ms.spin, false, n_src_old, n_dst_old);
  const int ts_src = net.per_site ? ms.src : 0, ts_dst = net.per_site ? ms.dst : 0;
  // z0' on S (lane = channel; two channels per lane when h > 32)
  for (int c = lane; c < h; c += 32) {
    for (int s = 0; s < nS; ++s) ms.feat[s][c] = sv.z0[(size_t)ms.site[s] * h + c];
    for (int p = 0; p < npairs; ++p) {
      const int s = ms.pair_s[p];
      if (s < 0) continue;
      const int d = p % kk;
      const bool from_src = p < kk;
      const int ts = from_src ? ts_src : ts_dst;
      const int nn = from_src ? n_src_new : n_dst_new;
      const int no = from_src ? n_src_old : n_dst_old;
      ms.feat[s][c] += net.KE[(((size_t)ts * 4 + nn) * kk + d) * h + c] - net.KE[(((size_t)ts * 4 + no) * kk + d) * h + c];
    }
    for (int s = 0; s < nS; ++s) {
      const int site = ms.site[s];
      if (z0_new) z0_new[s][c] = ms.feat[s][c];
      const T e = net.resid[0] ? net.embed[((size_t)(net.per_site ? site * 4 : 0) + ms.nnew[s]) * h + c] : T(0);
      ms.feat[s][c] = e + act_fn<T>(net.act, ms.feat[s][c]);
    }
  }
  __syncwarp();
  // site-wise layers 1..L-1: out[c] = res*in[c] + act(b[c] + sum_c' in[c'] W[c'][c])
  for (int l = 1; l < net.L; ++l) {
    const T* W = net.kernel[l];
    const T* bl = net.bias[l];
    const int res = net.resid[l];
    for (int s0 = 0; s0 < nS; s0 += 4) {
      const int ns = min(4, nS - s0);
      T acc[2][4];  // same summation order as the forward layer: bias first, then c' ascending
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int c = lane + 32 * u;
        const T b0 = (c < h) ? bl[c] : T(0);
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = b0;
      }
      for (int ci = 0; ci < h; ++ci) {
        T xin[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) xin[v] = (v < ns) ? ms.feat[s0 + v][ci] : T(0);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int c = lane + 32 * u;
          if (c < h) {
            const T w = W[(size_t)ci * h + c];
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] += xin[v] * w;
          }
        }
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int c = lane + 32 * u;
        if (c < h) {
#pragma unroll
          for (int v = 0; v < 4; ++v)
            if (v < ns) {
              const T prev = ms.feat[s0 + v][c];
              ms.feat[s0 + v][c] = (res ? prev : T(0)) + act_fn<T>(net.act, acc[u][v]);
            }
        }
      }
      __syncwarp();
    }
  }
  // Delta H
  for (int c = lane; c < h; c += 32)
    for (int s = 0; s < nS; ++s) ms.feat[s][c] -= sv.HL[(size_t)ms.site[s] * h + c];
  __syncwarp();
}

// Step 4: electron list on S after the move and the r x r matrix R. Returns r (valid in
// all lanes), or -1 when r exceeds kRMax.
template <typename T>
__device__ int move_matrix(const Lattice& lat, const Net<T>& net, const SampleView<T>& sv, MoveScratch<T>& ms) {
  const int lane = threadIdx.x & 31;
  const int N = lat.N, Ne = lat.Ne, h = net.h;
  if (lane == 0) {
    int r = 0;
    for (int s = 0; s < ms.nS; ++s)
      for (int sp = 0; sp < 2; ++sp) {
        if (!((ms.nnew[s] >> sp) & 1)) continue;
        const int site = ms.site[s];
        int slot, mv = 0;
        if ((ms.nold[s] >> sp) & 1) {
          slot = sv.slot_of_orb[sp * N + site];  // same electron, same orbital
        } else if (ms.kind == 0) {
          slot = sv.slot_of_orb[sp * N + ms.src];  // the hopping electron
          mv = 1;
        } else {
          slot = sv.slot_of_orb[sp * N + (site == ms.src ? ms.dst : ms.src)];  // exchanged spin
          mv = 1;
        }
        if (slot < 0) r = kRMax + 1;  // inconsistent slot map: reported as NaN
        if (r < kRMax) {
          ms.slot[r] = slot;
          ms.orb[r] = sp * N + site;
          ms.sidx[r] = s;
          ms.moved[r] = mv;
        }
        ++r;
      }
    ms.r = r;
  }
  __syncwarp();
  const int r = ms.r;
  if (r > kRMax) return -1;
  // base rows: identity for electrons that kept their orbital, G(o'_a, c_b) for moved ones.
  // G(o, c) = (M0[o] + proj_b[s]) . Binv[c] + H(L)_i . Pt[s][c]; the Ne-long dot products
  // are split over the lanes (coalesced rows of Binv) and reduced with shuffles.
  for (int a = 0; a < r; ++a) {
    if (!ms.moved[a]) {
      if (lane < r) ms.R[a][lane] = (a == lane) ? T(1) : T(0);
      continue;
    }
    const int o = ms.orb[a], sp = o / N, i = o - sp * N;
    const T* m0 = net.M0 + (size_t)o * Ne;
    const T* pb = net.proj_b + sp * Ne;
    const T* hl = sv.HL + (size_t)i * h;
    for (int bb = 0; bb < r; ++bb) {
      const int cb = ms.slot[bb];
      const T* brow = sv.Binv + (size_t)cb * Ne;
      const T* pt = sv.Pt + ((size_t)sp * Ne + cb) * h;
      T g = T(0);
      for (int k = lane; k < Ne; k += 32) g += (m0[k] + pb[k]) * brow[k];
      for (int c = lane; c < h; c += 32) g += hl[c] * pt[c];
      for (int off = 16; off > 0; off >>= 1) g += __shfl_xor_sync(0xffffffffu, g, off);
      if (lane == bb) ms.R[a][bb] = g;
    }
  }
  __syncwarp();
  // + Delta H_{s_a} . Pt[s_a][c_b], column b = lane
  if (lane < r) {
    const int cb = ms.slot[lane];
    for (int a = 0; a < r; ++a) {
      const int sp = ms.orb[a] / N;
      const T* pt = sv.Pt + ((size_t)sp * Ne + cb) * h;
      const T* dh = ms.feat[ms.sidx[a]];
      T v = T(0);
      for (int c = 0; c < h; ++c) v += dh[c] * pt[c];
      ms.R[a][lane] += v;
    }
  }
  __syncwarp();
  return r;
}

// Step 5: det of ms.R (r x r) by LU with partial pivoting, lane j owning column j.
// R is destroyed. Returns the determinant (same value in all lanes).
template <typename T>
__device__ T warp_det(MoveScratch<T>& ms, int r) {
  const int lane = threadIdx.x & 31;
  T det = T(1);
  for (int k = 0; k < r; ++k) {
    // pivot in column k, rows k..r-1 (lane k scans, broadcast)
    int p = k;
    if (lane == k) {
      T best = fabs(ms.R[k][k]);
      for (int i = k + 1; i < r; ++i) {
        const T v = fabs(ms.R[i][k]);
        if (v > best) {
          best = v;
          p = i;
        }
      }
    }
    p = __shfl_sync(0xffffffffu, p, k);
    if (p != k) {
      if (lane < r) {
        const T t = ms.R[k][lane];
        ms.R[k][lane] = ms.R[p][lane];
        ms.R[p][lane] = t;
      }
      det = -det;
    }
    __syncwarp();
    const T pv = ms.R[k][k];
    det *= pv;
    if (pv == T(0)) return T(0);
    if (lane > k && lane < r) {
      const T u = ms.R[k][lane];
      for (int i = k + 1; i < r; ++i) ms.R[i][lane] -= (ms.R[i][k] / pv) * u;
    }
    __syncwarp();
  }
  return det;
}

// Parity of the number of occupied orbitals strictly between o1 and o2 (Jordan-Wigner
// sign relating the slot-order ratio to the ascending-order ratio of a hop).
__device__ __forceinline__ int between_parity(const int8_t* occ, int N, int o1, int o2) {
  const int lo = min(o1, o2), hi = max(o1, o2);
  int cnt = 0;
  for (int o = lo + 1 + (threadIdx.x & 31); o < hi; o += 32) {
    const int s = o / N, i = o - s * N;
    cnt += (occ[i] >> s) & 1;
  }
  for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
  return cnt & 1;
}

}  // namespace scale
