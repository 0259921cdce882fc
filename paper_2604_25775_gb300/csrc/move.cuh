// move.cuh -- one connected configuration n -> n' handled by one warp (Sec. II.C).
//
//   1. touched sites T = {src, dst} ("exchange" set of Sec. II.C);
//   2. affected sites S = union over t in T of the layer-0 stencil around t (Eq. neighbor);
//      the later layers are site-wise, so S does not grow;
//   3. new features on S: layer-0 pre-activation z0' = z0 + sum over (t, d) of
//      KE[t][n'_t][d] - KE[t][n_t][d], then the residual / activation and the site-wise
//      layers (tensor cores in mixed mode: three TF32 products of a hi/lo split by default,
//      three BF16 products as an option; FP64 FMA in FP64 mode);
//   4. the electrons on S after the move, each with its determinant row (slot) c_a and new
//      orbital o'_a; the rank-r matrix of Eq. SMW with U = the changed rows,
//        R[a][b] = M'[o'_a] . Binv[c_b]
//                = delta_ab + (H'_{s_a} - H_{s_a}) . Pt[s_a][c_b]          (a kept its orbital)
//                = (M0[o'_a] + proj_b[s_a]) . Binv[c_b] + H'_{s_a} . Pt[s_a][c_b]   (a moved)
//      (the first term cached per walker as G0t[c_b][o'_a] and kept current by every commit)
//      is A = I_r + V^T Phi^-1 U with V^T = Phi'_C - Phi_C;
//   5. det R by LU with partial pivoting (lane j owns column j).
// det R is the slot-order ratio det Phi'/det Phi; the moved electrons keep their rows.
#pragma once

#include "mlp_mma.cuh"
#include "scale_internal.cuh"

namespace scale {

constexpr int kSMax = 18;  // affected sites for two touched sites and a 3x3 box or the 13-site plus
constexpr int kRMax = 32;  // electrons on the affected sites (lane per column)

template <typename T, int H>
struct MoveScratch {
  int nS, r, kind, src, dst, spin;
  int site[kSMax];
  int nold[kSMax], nnew[kSMax];
  int pair_s[2 * 13];  // S index of each (touched site, tap) pair, -1 if none (up to 13 taps)
  int slot[kRMax], orb[kRMax], sidx[kRMax], moved[kRMax];
  alignas(16) T feat[kSMax][H];   // new features H'(L) on S (tile loads/stores stop at nS)
  alignas(16) T hl[kSMax][H];     // cached features H(L) on S
  alignas(16) T R[kRMax][kRMax + 1];  // also the embedding rows of S while the features are built
};

// 16-byte asynchronous global -> shared copies (the warp waits for its own copies and then
// synchronises, after which every lane sees every row).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Per-sample views used by the move routines.
template <typename T>
struct SampleView {
  const int8_t* occ;           // [N] (shared memory copy)
  const int32_t* slot_of_orb;  // [2N]
  const T* z0;                 // [N][h]
  const T* HL;                 // [N][h]
  const T* Binv;               // [Ne][Ne]
  const T* Pt;                 // [2][Ne][h]
  const T* G0t;                // [Ne][2N]: (M0[o] + proj_b[s(o)]) . Binv[j]; null: not current
};

// Site-wise layer weights as hi/lo mma fragments, TF32 or BF16 by `kind` (mixed mode); null
// in FP64 mode.
struct MlpFrags {
  const WFrag* wf;
  int kind;             // kTF32, kFP16 or kBF16
  const float* oscale;  // kFP16: per-layer output factors (fp16_scales + kMaxLayers)
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

// Site-wise layers 1..L-1 on the rows of ms.feat (FP FMA path): lane = channel, four sites
// per pass, weights read through L1. Summation order: bias first, then c' ascending, the
// same as the forward layer kernel.
template <typename T, int H>
__device__ void mlp_simt(const Net<T>& net, MoveScratch<T, H>& ms, int nS) {
  const int lane = threadIdx.x & 31, h = net.h;
  for (int l = 1; l < net.L; ++l) {
    const T* W = net.kernel[l];
    const T* bl = net.bias[l];
    const int res = net.resid[l];
    for (int s0 = 0; s0 < nS; s0 += 4) {
      const int ns = min(4, nS - s0);
      T acc[2][4];
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
}

// Steps 1-3: S and the new last-layer features H'(L) on S in ms.feat, the cached H(L) in
// ms.hl. All lanes of the warp participate. z0_new (optional) receives z0' on S.
template <typename T, int H>
__device__ void move_features(const Lattice& lat, const Net<T>& net, int k0, const SampleView<T>& sv,
                              const MlpFrags& mf, MoveScratch<T, H>& ms, T (*z0_new)[H] = nullptr) {
  const int lane = threadIdx.x & 31;
  const int h = net.h, kk = net.taps0;  // taps of layer 0 (9 for the 3x3 box, 13 for the plus)
  const int npairs = 2 * kk;            // <= 32: one lane per pair
  // pairs (t, d): t = src (pair < kk) or dst; the site reached is t - offset(d)
  int s_site = -1;
  if (lane < npairs) {
    const int t = (lane < kk) ? ms.src : ms.dst;
    const int d = lane % kk;
    int dx, dy;
    stencil_tap(net.stencil, k0, d, dx, dy);
    s_site = site_off(lat, t, -dx, -dy);
  }
  const unsigned act_mask = __ballot_sync(0xffffffffu, s_site >= 0);
  const unsigned same = __match_any_sync(0xffffffffu, s_site);
  const int first = __ffs(same & act_mask) - 1;
  const bool is_first = (s_site >= 0) && (first == lane);
  const unsigned firsts = __ballot_sync(0xffffffffu, is_first);
  const int n_src_old = sv.occ[ms.src] & 3, n_dst_old = sv.occ[ms.dst] & 3;
  const int n_src_new = move_new_state(ms.kind, ms.spin, true, n_src_old, n_dst_old);
  const int n_dst_new = move_new_state(ms.kind, ms.spin, false, n_src_old, n_dst_old);
  if (s_site >= 0) {
    const int pos = __popc(firsts & ((1u << first) - 1u));
    ms.pair_s[lane] = pos;
    if (is_first) {
      ms.site[pos] = s_site;
      const int n_old = sv.occ[s_site] & 3;
      ms.nold[pos] = n_old;
      ms.nnew[pos] = (s_site == ms.src) ? n_src_new : (s_site == ms.dst) ? n_dst_new : n_old;
    }
  } else if (lane < npairs) {
    ms.pair_s[lane] = -1;
  }
  const int nS = __popc(firsts);
  if (lane == 0) ms.nS = nS;
  __syncwarp();
  const int ts_src = net.per_site ? ms.src : 0, ts_dst = net.per_site ? ms.dst : 0;
  // stage z0 and H(L) rows of S, add the layer-0 table deltas, activation + residual.
  constexpr bool kCopyRows = H <= 32 && kSMax * H <= kRMax * (kRMax + 1);
  if (kCopyRows && (h * (int)sizeof(T)) % 16 == 0) {
    // z0 -> feat, H(L) -> hl and the residual embedding rows -> the R area by asynchronous
    // 16-byte copies; the table-delta loads go out while they travel (two rounds of nine
    // touched pairs), so the staging costs about two memory round trips
    constexpr int E = 16 / (int)sizeof(T);
    const int cpr = h / E;  // chunks per row
    T* emb = &ms.R[0][0];   // [nS][h]
    const int nrows = nS * (net.resid[0] ? 3 : 2);
    for (int q = lane; q < nrows * cpr; q += 32) {
      const int row = q / cpr, v = q - row * cpr;
      const int part = row / nS, s = row - part * nS;
      const int site = ms.site[s];
      const T* src;
      T* dst;
      if (part == 0) {
        src = sv.z0 + (size_t)site * h;
        dst = ms.feat[s];
      } else if (part == 1) {
        src = sv.HL + (size_t)site * h;
        dst = ms.hl[s];
      } else {
        src = net.embed + ((size_t)(net.per_site ? site * 4 : 0) + ms.nnew[s]) * h;
        dst = emb + (size_t)s * h;
      }
      cp_async16(dst + v * E, src + v * E);
    }
    cp_async_commit();
    const int c = lane;
    const bool on_c = c < h;
#pragma unroll
    for (int p0 = 0; p0 < 27; p0 += 9) {  // the pairs in groups of nine (two groups for the box)
      if (p0 >= npairs) break;
      T kn[9], ko[9];
#pragma unroll
      for (int g = 0; g < 9; ++g) {
        const int p = p0 + g;
        kn[g] = ko[g] = T(0);
        if (on_c && p < npairs && ms.pair_s[p] >= 0) {
          const int d = p % kk;
          const bool from_src = p < kk;
          const int ts = from_src ? ts_src : ts_dst;
          const int nn = from_src ? n_src_new : n_dst_new;
          const int no = from_src ? n_src_old : n_dst_old;
          kn[g] = net.KE[(((size_t)ts * 4 + nn) * kk + d) * h + c];
          ko[g] = net.KE[(((size_t)ts * 4 + no) * kk + d) * h + c];
        }
      }
      if (p0 == 0) {
        cp_async_wait_all();
        __syncwarp();
      }
#pragma unroll
      for (int g = 0; g < 9; ++g) {
        const int p = p0 + g;
        if (on_c && p < npairs && ms.pair_s[p] >= 0) ms.feat[ms.pair_s[p]][c] += kn[g] - ko[g];
      }
    }
    if (on_c)
      for (int s = 0; s < nS; ++s) {
        const T zz = ms.feat[s][c];
        if (z0_new) z0_new[s][c] = zz;
        ms.feat[s][c] = (net.resid[0] ? emb[(size_t)s * h + c] : T(0)) + act_fn<T>(net.act, zz);
      }
  } else {
  // Loads are issued kG at a time into registers before any is used (groups predicated on
  // the actual counts): a handful of memory round trips instead of one per row.
  constexpr int kG = 6;
  for (int c = lane; c < h; c += 32) {
    // (a) z0 and H(L) rows of S
#pragma unroll 1
    for (int s0 = 0; s0 < nS; s0 += kG) {
      T z[kG], hv[kG];
#pragma unroll
      for (int g = 0; g < kG; ++g) {
        const bool on = s0 + g < nS;
        const int site = on ? ms.site[s0 + g] : 0;
        z[g] = on ? sv.z0[(size_t)site * h + c] : T(0);
        hv[g] = on ? sv.HL[(size_t)site * h + c] : T(0);
      }
#pragma unroll
      for (int g = 0; g < kG; ++g)
        if (s0 + g < nS) {
          ms.feat[s0 + g][c] = z[g];
          ms.hl[s0 + g][c] = hv[g];
        }
    }
    // (b) layer-0 table deltas of the touched (site, offset) pairs
#pragma unroll 1
    for (int p0 = 0; p0 < npairs; p0 += kG) {
      T kn[kG], ko[kG];
#pragma unroll
      for (int g = 0; g < kG; ++g) {
        const int p = p0 + g;
        kn[g] = ko[g] = T(0);
        if (p < npairs && ms.pair_s[p] >= 0) {
          const int d = p % kk;
          const bool from_src = p < kk;
          const int ts = from_src ? ts_src : ts_dst;
          const int nn = from_src ? n_src_new : n_dst_new;
          const int no = from_src ? n_src_old : n_dst_old;
          kn[g] = net.KE[(((size_t)ts * 4 + nn) * kk + d) * h + c];
          ko[g] = net.KE[(((size_t)ts * 4 + no) * kk + d) * h + c];
        }
      }
#pragma unroll
      for (int g = 0; g < kG; ++g) {
        const int p = p0 + g;
        if (p < npairs && ms.pair_s[p] >= 0) ms.feat[ms.pair_s[p]][c] += kn[g] - ko[g];
      }
    }
    // (c) activation + residual embedding
#pragma unroll 1
    for (int s0 = 0; s0 < nS; s0 += kG) {
      T ev[kG];
#pragma unroll
      for (int g = 0; g < kG; ++g) {
        const bool on = s0 + g < nS && net.resid[0];
        const int site = on ? ms.site[s0 + g] : 0;
        ev[g] = on ? net.embed[((size_t)(net.per_site ? site * 4 : 0) + ms.nnew[s0 + g]) * h + c] : T(0);
      }
#pragma unroll
      for (int g = 0; g < kG; ++g)
        if (s0 + g < nS) {
          const T zz = ms.feat[s0 + g][c];
          if (z0_new) z0_new[s0 + g][c] = zz;
          ms.feat[s0 + g][c] = ev[g] + act_fn<T>(net.act, zz);
        }
    }
  }
  }
  __syncwarp();
  if (net.L > 1) {
    if constexpr (sizeof(T) == 4 && H % 16 == 0) {
      if (mf.wf) {
        for (int r0t = 0; r0t < nS; r0t += 16) {
          float x[H / 8][4];
          tile_load<H>(x, &ms.feat[r0t][0], H, nS - r0t);
          if (mf.kind == kTF32)
            mlp_tile<H, kTF32>(x, mf.wf, net.bias, net.resid, net.L, net.act);
          else if (mf.kind == kFP16)
            mlp_tile<H, kFP16>(x, mf.wf, net.bias, net.resid, net.L, net.act, mf.oscale);
          else
            mlp_tile<H, kBF16>(x, mf.wf, net.bias, net.resid, net.L, net.act);
          __syncwarp();
          tile_store<H>(x, &ms.feat[r0t][0], H, nS - r0t);
        }
        __syncwarp();
        return;
      }
    }
    mlp_simt<T, H>(net, ms, nS);
  }
}

// Step 4: the electron list on S after the move and the r x r matrix R. Returns r (valid in
// all lanes), or -1 when r exceeds kRMax or a slot map is inconsistent.
// kDotFallback: sv.G0t may be null (a Metropolis commit), so the dot-product path is compiled
// in; the local-energy and ratio kernels always have the cache and leave it out.
template <typename T, int H, bool kDotFallback = false>
__device__ int move_matrix(const Lattice& lat, const Net<T>& net, const SampleView<T>& sv, MoveScratch<T, H>& ms) {
  const int lane = threadIdx.x & 31;
  const int N = lat.N, Ne = lat.Ne, h = net.h;
  const int nS = ms.nS;
  // electrons on S after the move: spin-up ones first, then spin-down, each group in S
  // order, compacted with ballots (the determinant does not depend on the row order
  // because rows and columns of R follow the same list)
  int r = 0, r_up = 0;
  bool bad = false;
  for (int sp = 0; sp < 2; ++sp) {
    if (sp == 1) r_up = r;
    for (int base = 0; base < nS; base += 32) {
      const int s = base + lane;
      int slot = -1, mv = 0;
      bool occ = false;
      if (s < nS) {
        occ = (ms.nnew[s] >> sp) & 1;
        if (occ) {
          const int site = ms.site[s];
          if ((ms.nold[s] >> sp) & 1) {
            slot = sv.slot_of_orb[sp * N + site];  // same electron, same orbital
          } else if (ms.kind == 0) {
            slot = sv.slot_of_orb[sp * N + ms.src];  // the hopping electron
            mv = 1;
          } else {
            slot = sv.slot_of_orb[sp * N + (site == ms.src ? ms.dst : ms.src)];  // exchanged spin
            mv = 1;
          }
        }
      }
      const unsigned bal = __ballot_sync(0xffffffffu, occ);
      if (occ) {
        const int pos = r + __popc(bal & ((1u << lane) - 1u));
        if (slot < 0) bad = true;
        if (pos < kRMax) {
          ms.slot[pos] = slot;
          ms.orb[pos] = sp * N + ms.site[s];
          ms.sidx[pos] = s;
          ms.moved[pos] = mv;
        }
      }
      r += __popc(bal);
    }
  }
  bad = __any_sync(0xffffffffu, bad);
  if (lane == 0) ms.r = r;
  __syncwarp();
  if (r > kRMax || bad) return -1;
  // Delta H in place of the cached rows: ms.hl[s] <- H'_s - H_s
  for (int c = lane; c < h; c += 32)
    for (int s = 0; s < nS; ++s) ms.hl[s][c] = ms.feat[s][c] - ms.hl[s][c];
  __syncwarp();
  const int cb = ms.slot[lane < r ? lane : 0];
  // Pt terms, column b = lane: the Pt[spin][c_b] row in registers (16 channels at a time),
  // each electron of that spin dotted against its feature row (H' if it moved, Delta H if
  // not); identity for the electrons that kept their orbital
  if constexpr (H <= 32) {
    if (r <= 16) {
      // two half-warps per column b = lane % 16, each with half of the Pt row in registers;
      // the halves meet in one shuffle (twice the active lanes of one column per lane)
      constexpr int HH = H / 2;
      const int bb = lane & 15, hc = lane >> 4;
      const int cbb = ms.slot[bb < r ? bb : 0];
      for (int sp = 0; sp < 2; ++sp) {
        const int a0 = sp ? r_up : 0, a1 = sp ? r : r_up;
        if (a0 == a1) continue;
        const T* pt = sv.Pt + ((size_t)sp * Ne + cbb) * h + hc * HH;
        T pv[HH];
#pragma unroll
        for (int u = 0; u < HH; ++u) pv[u] = (hc * HH + u < h) ? pt[u] : T(0);
        for (int a = a0; a < a1; ++a) {
          const T* row = (ms.moved[a] ? ms.feat[ms.sidx[a]] : ms.hl[ms.sidx[a]]) + hc * HH;
          T v[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
          for (int u = 0; u < HH; ++u)
            if (hc * HH + u < h) v[u & 3] += row[u] * pv[u];
          const T part = (v[0] + v[1]) + (v[2] + v[3]);
          const T tot = part + __shfl_xor_sync(0xffffffffu, part, 16);
          const T init = (!ms.moved[a] && a == bb) ? T(1) : T(0);
          if (hc == 0 && bb < r) ms.R[a][bb] = init + tot;
        }
      }
      __syncwarp();
    } else {
    // the whole Pt row of the lane's column in registers; every row of R written once
    for (int sp = 0; sp < 2; ++sp) {
      const int a0 = sp ? r_up : 0, a1 = sp ? r : r_up;
      if (a0 == a1) continue;
      const T* pt = sv.Pt + ((size_t)sp * Ne + cb) * h;
      T pv[H];
#pragma unroll
      for (int u = 0; u < H; ++u) pv[u] = (u < h) ? pt[u] : T(0);
      for (int a = a0; a < a1; ++a) {
        const T* row = ms.moved[a] ? ms.feat[ms.sidx[a]] : ms.hl[ms.sidx[a]];
        T v[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int u = 0; u < H; ++u)
          if (u < h) v[u & 3] += row[u] * pv[u];
        const T init = (!ms.moved[a] && a == lane) ? T(1) : T(0);
        if (lane < r) ms.R[a][lane] = init + ((v[0] + v[1]) + (v[2] + v[3]));
      }
    }
    __syncwarp();
    }
  } else {
  if (lane < r)
    for (int a = 0; a < r; ++a) ms.R[a][lane] = (!ms.moved[a] && a == lane) ? T(1) : T(0);
  __syncwarp();
  for (int sp = 0; sp < 2; ++sp) {
    const int a0 = sp ? r_up : 0, a1 = sp ? r : r_up;
    if (a0 == a1) continue;
    const T* pt = sv.Pt + ((size_t)sp * Ne + cb) * h;
    for (int c0 = 0; c0 < h; c0 += 16) {
      T pv[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) pv[u] = (c0 + u < h) ? pt[c0 + u] : T(0);
      for (int a = a0; a < a1; ++a) {
        const T* row = (ms.moved[a] ? ms.feat[ms.sidx[a]] : ms.hl[ms.sidx[a]]) + c0;
        T v0 = T(0), v1 = T(0);
#pragma unroll
        for (int u = 0; u < 16; u += 2) {
          if (c0 + u < h) v0 += row[u] * pv[u];
          if (c0 + u + 1 < h) v1 += row[u + 1] * pv[u + 1];
        }
        if (lane < r) ms.R[a][lane] += v0 + v1;
      }
    }
  }
  __syncwarp();
  }
  // moved rows: + (M0[o'] + proj_b[s]) . Binv[c_b] = G0t[c_b][o'], one cached entry per lane;
  // without the cache (a Metropolis sweep, which does not keep it current) the dot products
  // against the inverse, lanes split k, one warp reduction per b
  if (!kDotFallback || sv.G0t) {
    for (int a = 0; a < r; ++a) {
      if (!ms.moved[a]) continue;
      if (lane < r) ms.R[a][lane] += sv.G0t[(size_t)ms.slot[lane] * 2 * N + ms.orb[a]];
    }
  } else if constexpr (kDotFallback) {
    for (int a = 0; a < r; ++a) {
      if (!ms.moved[a]) continue;
      const T* m0b = net.M0b + (size_t)ms.orb[a] * Ne;
      constexpr int KK = 7;  // k values per lane per pass (224 per warp: one pass at 16x16)
      for (int b0 = 0; b0 < r; b0 += 4) {
        T g[4] = {T(0), T(0), T(0), T(0)};
        const T* br[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) br[q] = sv.Binv + (size_t)ms.slot[min(b0 + q, r - 1)] * Ne;
        for (int k0 = 0; k0 < Ne; k0 += 32 * KK) {
          T v[KK], bv[4][KK];
#pragma unroll
          for (int u = 0; u < KK; ++u) {
            const int k = k0 + lane + 32 * u;
            const bool on = k < Ne;
            v[u] = on ? m0b[k] : T(0);
#pragma unroll
            for (int q = 0; q < 4; ++q) bv[q][u] = on ? br[q][k] : T(0);
          }
#pragma unroll
          for (int u = 0; u < KK; ++u)
#pragma unroll
            for (int q = 0; q < 4; ++q) g[q] += v[u] * bv[q][u];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) g[q] += __shfl_xor_sync(0xffffffffu, g[q], off);
          if (lane == b0 + q && b0 + q < r) ms.R[a][lane] += g[q];
        }
      }
    }
  }
  __syncwarp();
  return r;
}

// 1/x rounded to nearest: the same value as the division 1/x, without its general path.
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }

// Pivot row of column k among rows [k, r) of R (lane i holds row i): the largest |R[i][k]|,
// ties to the lowest row. Same value in every lane.
template <typename T>
__device__ __forceinline__ int warp_pivot(const T (*R)[kRMax + 1], int k, int r) {
  const int lane = threadIdx.x & 31;
  const bool mine = lane >= k && lane < r;
  if constexpr (sizeof(T) == 4) {
    // |x| of non-negative floats orders like its bit pattern: one warp max + ballot
    const unsigned key = mine ? __float_as_uint(fabsf((float)R[lane][k])) : 0u;
    const unsigned mx = __reduce_max_sync(0xffffffffu, key);
    return __ffs(__ballot_sync(0xffffffffu, mine && key == mx)) - 1;
  } else {
    T best = mine ? fabs(R[lane][k]) : T(-1);
    int p = lane;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const T ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int op = __shfl_xor_sync(0xffffffffu, p, off);
      if (ob > best || (ob == best && op < p)) {
        best = ob;
        p = op;
      }
    }
    return p;
  }
}

// Step 5: det of R (r x r, r <= kRMax) by LU with partial pivoting, lane j owning column j;
// the pivot search is a warp argmax over the rows, one reciprocal per column. R is destroyed.
// Returns the determinant (same value in all lanes).
template <typename T>
__device__ T warp_det_R(T (*R)[kRMax + 1], int r) {
  const int lane = threadIdx.x & 31;
  T det = T(1);
  for (int k = 0; k < r; ++k) {
    const int p = warp_pivot<T>(R, k, r);
    if (p != k) {
      if (lane < r) {
        const T t = R[k][lane];
        R[k][lane] = R[p][lane];
        R[p][lane] = t;
      }
      det = -det;
    }
    __syncwarp();
    const T pv = R[k][k];
    det *= pv;
    if (pv == T(0)) return T(0);
    const T inv = recip(pv);
    // multipliers in column k (lane i > k), then the trailing update (lane j > k)
    if (lane > k && lane < r) R[lane][k] *= inv;
    __syncwarp();
    if (lane > k && lane < r) {
      const T u = R[k][lane];
      for (int i = k + 1; i < r; ++i) R[i][lane] -= R[i][k] * u;
    }
    __syncwarp();
  }
  return det;
}

template <typename T, int H>
__device__ T warp_det(MoveScratch<T, H>& ms, int r) {
  return warp_det_R<T>(ms.R, r);
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
