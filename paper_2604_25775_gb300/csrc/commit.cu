// commit.cu -- accept one move per sample: Sherman-Morrison-Woodbury update of the cached
// inverse (Eq. SMW, second line), rank-r update of the projector, incremental update of
// the cached features, occupations and slot maps, running log|det|, and the drift check
// that schedules an FP64 re-factorisation.
//
// With R = Phi'_C Phi^-1[:, C] (the capacitance matrix I_r + V^T Phi^-1 U of Eq. SMW for
// the changed rows C) and X = Phi'_C Phi^-1 - E_C^T (r x Ne),
//     Phi'^-1 = Phi^-1 - Phi^-1[:, C] R^-1 X,
// i.e. in the dual-row layout Binv[j] <- Binv[j] - sum_b D[b][j] Binv[c_b], D = R^-1 X,
// and the projector, linear in Binv[j], takes the same update.
#include <algorithm>

#include "move.cuh"

namespace scale {

namespace {

struct CommitArgs {
  Lattice lat;
  int k0;
  int8_t* occ;
  int32_t* slot_of_orb;
  int32_t* orb_of_slot;
  void* z0;
  void* HL;
  void* Binv;
  void* Pt;
  void* G0t;
  double* logabs;
  int32_t* sign_slot;
  int32_t* status;
  int32_t* commits;
  double* drift;
  double drift_tol;
  const int32_t* moves;
  void* scratch;          // [B][commit_scratch_elems] T: D, saved Binv rows, saved G0t rows
  unsigned long long* drift_max_bits;
  int32_t* n_commits;
  MlpFrags mf;
  // Metropolis mode (pick != null): the move of sample b is the hop of its pick[b]-th
  // occupied orbital (ascending o = s*N + i) along direction dir[b] (+x, -x, +y, -y),
  // accepted when u[b] < |psi(n')/psi(n)|^2 = (det R)^2; accepted[b] counts acceptances.
  const int32_t* pick;
  const int32_t* dir;
  const double* u;
  int32_t* accepted;
};

constexpr int kCommitThreads = 256;
constexpr int kCommitWarps = kCommitThreads / 32;

// In-place inverse of the r x r matrix R (warp; lane j owns column j of R and of Ri),
// Gauss-Jordan with partial pivoting and explicit row swaps. Each step reads the pivot
// column once into registers (one value per lane) and eliminates every other row from
// shuffled multipliers, so the row loop carries no warp barrier. Returns the determinant.
template <typename T>
__device__ T warp_inverse(T (*R)[kRMax + 1], T (*Ri)[kRMax + 1], int r) {
  const int lane = threadIdx.x & 31;
  if (lane < r)
    for (int i = 0; i < r; ++i) Ri[i][lane] = (i == lane) ? T(1) : T(0);
  __syncwarp();
  T det = T(1);
  for (int k = 0; k < r; ++k) {
    const int p = warp_pivot<T>(R, k, r);
    if (p != k) {
      if (lane < r) {
        T t = R[k][lane]; R[k][lane] = R[p][lane]; R[p][lane] = t;
        t = Ri[k][lane]; Ri[k][lane] = Ri[p][lane]; Ri[p][lane] = t;
      }
      det = -det;
    }
    __syncwarp();
    const T pv = R[k][k];
    det *= pv;
    if (pv == T(0)) return T(0);
    const T inv = recip(pv);
    T rk = T(0), rik = T(0), f = T(0);
    if (lane < r) {
      rk = R[k][lane] * inv;
      rik = Ri[k][lane] * inv;
      f = R[lane][k];
    }
    __syncwarp();
    if (lane < r) {
      R[k][lane] = rk;
      Ri[k][lane] = rik;
    }
    for (int i = 0; i < r; ++i) {
      const T fi = __shfl_sync(0xffffffffu, f, i);
      if (i != k && lane < r) {
        R[i][lane] -= fi * rk;
        Ri[i][lane] -= fi * rik;
      }
    }
    __syncwarp();
  }
  return det;
}

// Four consecutive elements (16-byte aligned for float, 32-byte for double).
__device__ __forceinline__ void load4(const float* p, float v[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4(const double* p, double v[4]) {
  const double2 q0 = reinterpret_cast<const double2*>(p)[0], q1 = reinterpret_cast<const double2*>(p)[1];
  v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}

// 16-byte vectors: four floats or two doubles.
__device__ __forceinline__ void vld(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void vld(const double* p, double (&v)[2]) {
  const double2 q = *reinterpret_cast<const double2*>(p);
  v[0] = q.x; v[1] = q.y;
}
__device__ __forceinline__ void vst(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void vst(double* p, const double (&v)[2]) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
}

// Shared-memory layout of k_commit, every region 16-byte aligned. The saved rows Bc and
// the matrix D sit in shared memory when they fit (flags), else in the sample's scratch.
struct CommitSmem {
  size_t ms, z0n, Ri, Y, Pc, g, nrm, bc, d, slot, occ, total;
};
template <typename T, int H>
__host__ __device__ inline CommitSmem commit_smem(int N, int NeP, bool bc_smem, bool d_smem) {
  CommitSmem s{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = (off + bytes + 15) & ~size_t(15);
    return at;
  };
  s.ms = take(sizeof(MoveScratch<T, H>));
  s.z0n = take(sizeof(T) * kSMax * H);
  s.Ri = take(sizeof(T) * kRMax * (kRMax + 1));
  s.Y = take(sizeof(T) * 2 * kRMax * H);
  s.Pc = take(sizeof(T) * 2 * kRMax * H);
  s.g = take(sizeof(T) * 2 * NeP);
  s.nrm = take(sizeof(T) * 2 * kRMax);
  s.bc = bc_smem ? take(sizeof(T) * kRMax * NeP) : 0;
  s.d = d_smem ? take(sizeof(T) * kRMax * NeP) : 0;
  s.slot = take(sizeof(int32_t) * 2 * N);
  s.occ = take(N);
  s.total = off;
  return s;
}

// One CTA per sample.
//  (A) warp 0: receptive-field update of the move (new layer-0 pre-activations z0', new
//      features H'(L) and Delta H on S), the r x r capacitance matrix R and its inverse.
//      Meanwhile warps 1.. form g_m[j] = (M0[o'_m] + proj_b) . Binv[j] for the moved
//      orbitals o'_m and every slot j (the part of G(o'_m, j) that needs all of Binv).
//  (B) X = Phi'_C Phi^-1 - E_C^T is never stored: with u_a = Delta H (unmoved row) or
//      H' (moved row) of the electron's site and s_a its spin,
//          X[a][j] = u_a . Pt[s_a][j] + [a moved] (g(a)[j] - delta_{j c_a}),
//      so D = R^-1 X = sum_s Y_s Pt[s]^T + R^-1 (moved part), with the small
//      Y_s[b][c] = sum_{a: s_a = s} (R^-1)[b][a] u_a[c].
//  (C) Binv[j] -= sum_b D[b][j] Binv_old[c_b] and Pt[s][j] -= sum_b D[b][j] Pt_old[s][c_b],
//      four rows j per thread, lanes along the row.
//  (D) features, occupations, slot maps, log|det|, and the drift check.
// A capacitance determinant that is zero or not finite (or a sample whose Phi was
// singular) cannot take the Woodbury step: the move is applied to the occupations only and
// the sample is re-factorised in FP64 within the same call.
template <typename T, int H>
__global__ void __launch_bounds__(kCommitThreads, 2) k_commit(CommitArgs a, Net<T> net, int bc_in_smem, int d_in_smem) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = a.lat.N, Ne = a.lat.Ne, h = net.h;
  const int NeP = (Ne + 3) & ~3;
  const CommitSmem L = commit_smem<T, H>(N, NeP, bc_in_smem, d_in_smem);
  MoveScratch<T, H>& ms = *reinterpret_cast<MoveScratch<T, H>*>(smem + L.ms);
  T(*z0n)[H] = reinterpret_cast<T(*)[H]>(smem + L.z0n);               // [kSMax][H]
  T(*Ri)[kRMax + 1] = reinterpret_cast<T(*)[kRMax + 1]>(smem + L.Ri);  // [kRMax][kRMax+1]
  T(*Y)[kRMax][H] = reinterpret_cast<T(*)[kRMax][H]>(smem + L.Y);     // [2][kRMax][H]
  T(*Pc)[kRMax][H] = reinterpret_cast<T(*)[kRMax][H]>(smem + L.Pc);   // [2][kRMax][H]
  T* g = reinterpret_cast<T*>(smem + L.g);                            // [2][NeP]
  T* nrm = reinterpret_cast<T*>(smem + L.nrm);                        // [2 kRMax] squared row norms
  int32_t* slot_s = reinterpret_cast<int32_t*>(smem + L.slot);
  int8_t* occ_s = reinterpret_cast<int8_t*>(smem + L.occ);
  __shared__ int s_go;
  __shared__ double s_det;
  __shared__ unsigned long long s_drift_bits;

  const int b = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int st = a.status[b];
  if (st & (SCALE_SAMPLE_BAD_COUNT | SCALE_SAMPLE_DOUBLE_OCC)) return;
  const bool metropolis = a.pick != nullptr;
  int kind = -1, src = 0, dst = 0, spin = 0;
  if (!metropolis) {
    const int32_t* mv = a.moves + (size_t)b * 4;
    kind = mv[0];
    src = mv[1];
    dst = mv[2];
    spin = mv[3];
    if (kind < 0) return;
  }
  for (int i = tid; i < N; i += kCommitThreads) occ_s[i] = a.occ[(size_t)b * N + i];
  for (int o = tid; o < 2 * N; o += kCommitThreads) slot_s[o] = a.slot_of_orb[(size_t)b * 2 * N + o];
  __syncthreads();
  if (metropolis) {
    // proposal: the pick-th occupied orbital in ascending order, one site along dir
    __shared__ int s_mv[4];
    if (warp == 0) {
      int k = a.pick[b], o_src = -1;
      for (int o0 = 0; o0 < 2 * N && o_src < 0 && k >= 0; o0 += 32) {
        const int o = o0 + lane;
        const int s = o >= N ? 1 : 0;
        const bool on = o < 2 * N && ((occ_s[o - s * N] >> s) & 1);
        const unsigned m = __ballot_sync(0xffffffffu, on);
        const int cnt = __popc(m);
        if (k < cnt) o_src = o0 + (int)__fns(m, 0, k + 1);
        else k -= cnt;
      }
      if (lane == 0) {
        const int d = a.dir[b];
        int j = -1, s = 0, i = 0;
        if (o_src >= 0 && d >= 0 && d < 4) {
          s = o_src >= N ? 1 : 0;
          i = o_src - s * N;
          j = site_off(a.lat, i, d == 0 ? 1 : (d == 1 ? -1 : 0), d == 2 ? 1 : (d == 3 ? -1 : 0));
        }
        s_mv[0] = j >= 0 ? 0 : -1;
        s_mv[1] = i;
        s_mv[2] = j;
        s_mv[3] = s;
      }
    }
    __syncthreads();
    kind = s_mv[0];
    src = s_mv[1];
    dst = s_mv[2];
    spin = s_mv[3];
    if (kind < 0) return;  // off an open edge
  }
  if (!move_allowed(a.lat, kind, src, dst, spin, occ_s)) return;  // uniform across the CTA
  const bool singular = st & SCALE_SAMPLE_SINGULAR;
  const int n_src = occ_s[src], n_dst = occ_s[dst];
  // moved orbitals (destination rows of the moved electrons)
  int n_moved, om0, om1 = -1;
  if (kind == 0) {
    n_moved = 1;
    om0 = spin * N + dst;
  } else {
    const int s_up = (n_src == 1) ? 0 : 1;  // spin on src before the exchange
    n_moved = 2;
    om0 = s_up * N + dst;
    om1 = (1 - s_up) * N + src;
  }

  T* zb = (T*)a.z0 + (size_t)b * N * h;
  T* hb = (T*)a.HL + (size_t)b * N * h;
  T* Bb = (T*)a.Binv + (size_t)b * Ne * Ne;
  T* Pb = (T*)a.Pt + (size_t)b * 2 * Ne * h;
  const int No = 2 * N;
  T* Gb = (T*)a.G0t + (size_t)b * Ne * No;
  T* scr = (T*)a.scratch + (size_t)b * commit_scratch_elems(Ne, N);
  T* D = d_in_smem ? reinterpret_cast<T*>(smem + L.d) : scr;                         // [kRMax][NeP]
  T* Bc = bc_in_smem ? reinterpret_cast<T*>(smem + L.bc) : scr + (size_t)kRMax * NeP;  // [kRMax][NeP]
  T* Gc = scr + (size_t)2 * kRMax * NeP;                                               // [kRMax][2N]

  SampleView<T> sv;
  sv.occ = occ_s;
  sv.slot_of_orb = slot_s;
  sv.z0 = zb;
  sv.HL = hb;
  sv.Binv = Bb;
  sv.Pt = Pb;
  sv.G0t = metropolis ? nullptr : Gb;  // a sweep does not keep G0t current
  if (warp == 0) {
    if (lane == 0) {
      ms.kind = kind;
      ms.src = src;
      ms.dst = dst;
      ms.spin = spin;
    }
    __syncwarp();
    move_features<T, H>(a.lat, net, a.k0, sv, a.mf, ms, z0n);
    const int r = move_matrix<T, H, true>(a.lat, net, sv, ms);
    T det = T(0);
    if (r > 0 && !singular) det = warp_inverse<T>(ms.R, Ri, r);
    if (lane == 0) {
      // 1: Woodbury step; 2: occupations only, re-factorised in FP64 in this call; 0: nothing
      const bool ok = r > 0 && !singular && det != T(0) && isfinite((double)det);
      int go;
      if (!metropolis) {
        go = ok ? 1 : 2;
      } else if (singular) {
        go = 2;  // psi(n) = 0: every move is accepted
      } else if (r <= 0 || !isfinite((double)det)) {
        go = 0;  // ratio not available: rejected, the sample is re-factorised
        a.status[b] |= SCALE_SAMPLE_DRIFT;
      } else {
        go = a.u[b] < (double)det * (double)det ? 1 : 0;
      }
      s_go = go;
      s_det = (double)det;
      s_drift_bits = 0ull;
    }
  } else if (!singular && !metropolis) {
    // g_m[j] = (M0[o'_m] + proj_b) . Binv[j] for the moved orbitals: the cached G0t column
    for (int q = tid - 32; q < n_moved * Ne; q += kCommitThreads - 32) {
      const int m = q / Ne, j = q - m * Ne;
      g[m * NeP + j] = Gb[(size_t)j * No + (m ? om1 : om0)];
    }
  } else if (!singular) {
    // a Metropolis sweep does not keep G0t current (scale_sweep rebuilds it at the end): the
    // dot products against the inverse, four slots j per pass, lanes along k, every load of a
    // pass in flight before the first use
    constexpr int KU = 32 / sizeof(T);  // k values per lane per pass
    for (int m = 0; m < n_moved; ++m) {
      const T* m0b = net.M0b + (size_t)(m ? om1 : om0) * Ne;
      for (int j0 = 4 * (warp - 1); j0 < Ne; j0 += 4 * (kCommitWarps - 1)) {
        T v[4] = {T(0), T(0), T(0), T(0)};
        for (int k0 = 0; k0 < Ne; k0 += 32 * KU) {
          T x[KU], y[4][KU];
#pragma unroll
          for (int u = 0; u < KU; ++u) {
            const int k = k0 + lane + 32 * u;
            const bool on = k < Ne;
            x[u] = on ? m0b[k] : T(0);
#pragma unroll
            for (int i = 0; i < 4; ++i) y[i][u] = (on && j0 + i < Ne) ? Bb[(size_t)(j0 + i) * Ne + k] : T(0);
          }
#pragma unroll
          for (int u = 0; u < KU; ++u)
#pragma unroll
            for (int i = 0; i < 4; ++i) v[i] += x[u] * y[i][u];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          T sum = v[i];
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
          if (lane == 0 && j0 + i < Ne) g[m * NeP + j0 + i] = sum;
        }
      }
    }
  }
  __syncthreads();

  if (s_go == 0) return;
  if (s_go == 2) {
    // no Woodbury step: apply the move to the occupations, re-factorise in this call
    if (tid == 0) {
      a.occ[(size_t)b * N + src] = (int8_t)move_new_state(kind, spin, true, n_src, n_dst);
      a.occ[(size_t)b * N + dst] = (int8_t)move_new_state(kind, spin, false, n_src, n_dst);
      a.status[b] |= SCALE_SAMPLE_DRIFT;
      a.commits[b] += 1;
      atomicAdd(a.n_commits, 1);
      if (metropolis) a.accepted[b] += 1;
    }
    return;
  }
  const int r = ms.r;

  constexpr int V = 16 / sizeof(T);  // elements per 16-byte vector
  const bool vrow = (Ne % V) == 0;   // Binv rows are 16-byte aligned
  const bool vh = (h % V) == 0;      // Pt rows are 16-byte aligned
  const int nquad = (Ne + 3) >> 2;

  // (B1) old rows Binv[c_b], Pt[s][c_b]; Y_s = R^-1 restricted to spin-s rows times u
  for (int bi = warp; bi < r; bi += kCommitWarps) {
    const T* src_row = Bb + (size_t)ms.slot[bi] * Ne;
    T* dst_row = Bc + (size_t)bi * NeP;
    if (vrow) {
      for (int kv = lane; kv < Ne / V; kv += 32) {
        T v[V];
        vld(src_row + kv * V, v);
        vst(dst_row + kv * V, v);
      }
    } else {
      for (int k = lane; k < Ne; k += 32) dst_row[k] = src_row[k];
    }
  }
  if (!metropolis)
    for (int q = tid; q < r * No; q += kCommitThreads) {  // old G0t rows of the slots c_b
      const int bi = q / No, o = q - bi * No;
      Gc[q] = Gb[(size_t)ms.slot[bi] * No + o];
    }
  for (int q = tid; q < 2 * kRMax * H; q += kCommitThreads) {
    const int sp = q / (kRMax * H), rem = q - sp * kRMax * H, bi = rem / H, c = rem - bi * H;
    T pc = T(0), y = T(0);
    if (bi < r && c < h) {
      pc = Pb[((size_t)sp * Ne + ms.slot[bi]) * h + c];
      for (int ai = 0; ai < r; ++ai) {
        if ((ms.orb[ai] >= N ? 1 : 0) != sp) continue;
        const T u = ms.moved[ai] ? ms.feat[ms.sidx[ai]][c] : ms.hl[ms.sidx[ai]][c];
        y += Ri[bi][ai] * u;
      }
    }
    Pc[sp][bi][c] = pc;
    Y[sp][bi][c] = y;
  }
  __syncthreads();

  // (B2) D[b][j], one slot j and eight rows b per item; the 2h projector values of slot j
  // are fetched with all their loads in flight before the first use
  const int nbg = (r + 7) >> 3;
  for (int q = tid; q < nbg * Ne; q += kCommitThreads) {
    const int bg = q / Ne, j = q - bg * Ne, b0 = bg * 8;
    T acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = T(0);
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      const T* pt = Pb + ((size_t)sp * Ne + j) * h;
      if (vh) {
        constexpr int kCV = (H < 32 ? H : 32) / V;  // vectors of projector values in flight
#pragma unroll 1
        for (int c0 = 0; c0 < h; c0 += kCV * V) {
          T p[kCV][V];
#pragma unroll
          for (int cv = 0; cv < kCV; ++cv)
            if (c0 + cv * V < h) vld(pt + c0 + cv * V, p[cv]);
#pragma unroll
          for (int cv = 0; cv < kCV; ++cv)
            if (c0 + cv * V < h) {
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                T y[V];
                vld(&Y[sp][b0 + u][c0 + cv * V], y);  // rows >= r of Y are zero
#pragma unroll
                for (int v = 0; v < V; ++v) acc[u] += y[v] * p[cv][v];
              }
            }
        }
      } else {
        for (int c = 0; c < h; ++c) {
          const T pv = pt[c];
#pragma unroll
          for (int u = 0; u < 8; ++u) acc[u] += Y[sp][b0 + u][c] * pv;
        }
      }
    }
    for (int ai = 0; ai < r; ++ai) {
      if (!ms.moved[ai]) continue;
      const int m = (ms.orb[ai] == om0) ? 0 : 1;
      const T gv = g[m * NeP + j] - (j == ms.slot[ai] ? T(1) : T(0));
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (b0 + u < r) acc[u] += Ri[b0 + u][ai] * gv;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (b0 + u < r) D[(size_t)(b0 + u) * NeP + j] = acc[u];
  }
  // pad columns Ne..NeP-1 of the rows read below are zero
  for (int q = tid; q < r * (NeP - Ne); q += kCommitThreads) {
    const int bi = q / (NeP - Ne), j = Ne + q - bi * (NeP - Ne);
    D[(size_t)bi * NeP + j] = T(0);
  }
  __syncthreads();

  // (C1) Binv[j][k] -= sum_b D[b][j] Bc[b][k]: a 4-row x V-column register tile per thread,
  // lanes along the row; per b one vector of Bc and one of D, 4V multiply-adds
  if (vrow) {
    const int nkv = Ne / V, nkc = (nkv + 31) >> 5;
    for (int tile = warp; tile < nquad * nkc; tile += kCommitWarps) {
      const int jq = tile / nkc, kc = tile - jq * nkc, j0 = 4 * jq, kv = kc * 32 + lane;
      if (kv >= nkv) continue;
      T acc[4][V];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (j0 + i < Ne) {
          vld(Bb + (size_t)(j0 + i) * Ne + kv * V, acc[i]);
        } else {
#pragma unroll
          for (int v = 0; v < V; ++v) acc[i][v] = T(0);
        }
      }
#pragma unroll 2
      for (int bi = 0; bi < r; ++bi) {
        T bc[V], d[4];
        vld(Bc + (size_t)bi * NeP + kv * V, bc);
        load4(D + (size_t)bi * NeP + j0, d);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int v = 0; v < V; ++v) acc[i][v] -= d[i] * bc[v];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (j0 + i < Ne) vst(Bb + (size_t)(j0 + i) * Ne + kv * V, acc[i]);
    }
  } else {
    for (int j0 = 4 * warp; j0 < Ne; j0 += 4 * kCommitWarps) {
      for (int k = lane; k < Ne; k += 32) {
        T acc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] = (j0 + i < Ne) ? Bb[(size_t)(j0 + i) * Ne + k] : T(0);
        for (int bi = 0; bi < r; ++bi) {
          const T bc = Bc[(size_t)bi * NeP + k];
          T d[4];
          load4(D + (size_t)bi * NeP + j0, d);
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[i] -= d[i] * bc;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (j0 + i < Ne) Bb[(size_t)(j0 + i) * Ne + k] = acc[i];
      }
    }
  }
  // (C2) Pt[s][j][c] -= sum_b D[b][j] Pc[s][b][c]: a 4-row x V-channel tile per thread
  if (vh) {
    const int ncv = h / V;
    for (int q = tid; q < 2 * nquad * ncv; q += kCommitThreads) {
      const int cv = q % ncv, rest = q / ncv, jq = rest % nquad, sp = rest / nquad, j0 = 4 * jq;
      T* prow = Pb + (size_t)sp * Ne * h;
      T acc[4][V];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (j0 + i < Ne) {
          vld(prow + (size_t)(j0 + i) * h + cv * V, acc[i]);
        } else {
#pragma unroll
          for (int v = 0; v < V; ++v) acc[i][v] = T(0);
        }
      }
#pragma unroll 2
      for (int bi = 0; bi < r; ++bi) {
        T pc[V], d[4];
        vld(&Pc[sp][bi][cv * V], pc);
        load4(D + (size_t)bi * NeP + j0, d);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int v = 0; v < V; ++v) acc[i][v] -= d[i] * pc[v];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (j0 + i < Ne) vst(prow + (size_t)(j0 + i) * h + cv * V, acc[i]);
    }
  } else {
    for (int q = tid; q < 2 * nquad * h; q += kCommitThreads) {
      const int c = q % h, rest = q / h, jq = rest % nquad, sp = rest / nquad, j0 = 4 * jq;
      T* prow = Pb + (size_t)sp * Ne * h;
      T acc[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i] = (j0 + i < Ne) ? prow[(size_t)(j0 + i) * h + c] : T(0);
      for (int bi = 0; bi < r; ++bi) {
        const T pc = Pc[sp][bi][c];
        T d[4];
        load4(D + (size_t)bi * NeP + j0, d);
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] -= d[i] * pc;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (j0 + i < Ne) prow[(size_t)(j0 + i) * h + c] = acc[i];
    }
  }
  // (C3) G0t[j][o] -= sum_b D[b][j] Gc[b][o]: G0t[j] = (M0 + proj_b) Binv[j] is linear in
  // Binv[j], so it takes the same rank-r step; a 4-row x V-column tile per thread (not in a
  // Metropolis sweep, which rebuilds G0t once at its end)
  if (metropolis) {
  } else if (No % V == 0) {
    // two tiles per thread (rows j0.. and j0 + 4..), both loaded before the updates: twice the
    // bytes in flight per thread of this streaming step
    const int nov = No / V, ntile = nquad * nov;
    for (int q = tid; q < ntile; q += 2 * kCommitThreads) {
      const int q2 = q + kCommitThreads;
      const bool two = q2 < ntile;
      const int ov = q % nov, j0 = 4 * (q / nov);
      const int ov2 = two ? q2 % nov : ov, j02 = two ? 4 * (q2 / nov) : j0;
      T acc[2][4][V];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int jj = t ? j02 : j0, oo = t ? ov2 : ov;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (jj + i < Ne && (t == 0 || two)) {
            vld(Gb + (size_t)(jj + i) * No + oo * V, acc[t][i]);
          } else {
#pragma unroll
            for (int v = 0; v < V; ++v) acc[t][i][v] = T(0);
          }
        }
      }
#pragma unroll 2
      for (int bi = 0; bi < r; ++bi) {
        T gc[2][V], d[2][4];
        vld(Gc + (size_t)bi * No + ov * V, gc[0]);
        load4(D + (size_t)bi * NeP + j0, d[0]);
        vld(Gc + (size_t)bi * No + ov2 * V, gc[1]);
        load4(D + (size_t)bi * NeP + j02, d[1]);
#pragma unroll
        for (int t = 0; t < 2; ++t)
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int v = 0; v < V; ++v) acc[t][i][v] -= d[t][i] * gc[t][v];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (j0 + i < Ne) vst(Gb + (size_t)(j0 + i) * No + ov * V, acc[0][i]);
      if (two) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (j02 + i < Ne) vst(Gb + (size_t)(j02 + i) * No + ov2 * V, acc[1][i]);
      }
    }
  } else {
    for (int q = tid; q < nquad * No; q += kCommitThreads) {
      const int o = q % No, j0 = 4 * (q / No);
      T acc[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i] = (j0 + i < Ne) ? Gb[(size_t)(j0 + i) * No + o] : T(0);
      for (int bi = 0; bi < r; ++bi) {
        const T gc = Gc[(size_t)bi * No + o];
        T d[4];
        load4(D + (size_t)bi * NeP + j0, d);
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] -= d[i] * gc;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (j0 + i < Ne) Gb[(size_t)(j0 + i) * No + o] = acc[i];
    }
  }
  // (D) features on S: z0 <- z0', H(L) <- H'(L)
  for (int q = tid; q < ms.nS * h; q += kCommitThreads) {
    const int s = q / h, c = q - s * h;
    const int site = ms.site[s];
    zb[(size_t)site * h + c] = z0n[s][c];
    hb[(size_t)site * h + c] = ms.feat[s][c];
  }
  if (tid == 0) {
    // occupations and slot maps: moved electrons keep their rows
    if (kind == 0) {
      const int slot = slot_s[spin * N + src];
      a.slot_of_orb[(size_t)b * 2 * N + spin * N + src] = -1;
      a.slot_of_orb[(size_t)b * 2 * N + spin * N + dst] = slot;
      a.orb_of_slot[(size_t)b * Ne + slot] = spin * N + dst;
    } else {
      const int s_up = (n_src == 1) ? 0 : 1;
      const int s_dn = 1 - s_up;
      const int slot1 = slot_s[s_up * N + src], slot2 = slot_s[s_dn * N + dst];
      a.slot_of_orb[(size_t)b * 2 * N + s_up * N + src] = -1;
      a.slot_of_orb[(size_t)b * 2 * N + s_dn * N + dst] = -1;
      a.slot_of_orb[(size_t)b * 2 * N + s_up * N + dst] = slot1;
      a.slot_of_orb[(size_t)b * 2 * N + s_dn * N + src] = slot2;
      a.orb_of_slot[(size_t)b * Ne + slot1] = s_up * N + dst;
      a.orb_of_slot[(size_t)b * Ne + slot2] = s_dn * N + src;
    }
    a.occ[(size_t)b * N + src] = (int8_t)move_new_state(kind, spin, true, n_src, n_dst);
    a.occ[(size_t)b * N + dst] = (int8_t)move_new_state(kind, spin, false, n_src, n_dst);
    a.logabs[b] += log(fabs(s_det));
    if (s_det < 0) a.sign_slot[b] = -a.sign_slot[b];
    a.commits[b] += 1;
    atomicAdd(a.n_commits, 1);
    if (metropolis) a.accepted[b] += 1;
  }
  __syncthreads();
  // Drift check on the changed rows: the normalised residual
  //   max_{a,b} | M'[o'_a] . Binv'[c_b] - delta_ab | / (|M'[o'_a]|_2 |Binv'[c_b]|_2)
  // with M'[o'] = M0[o'] + proj_b[s] + H'(L)_i W_s built from the new features. Each dot
  // is split over the lanes (about Ne/32 terms each) and summed by a 5-level tree, so its
  // rounding error is at most about (Ne/32 + 5) units of the working precision relative to
  // |M'||Binv'| -- for Ne <= 896 in FP32 under 2e-6, far below any useful tolerance.
  // Normalised this way a freshly rounded inverse sits near the working precision whatever
  // the conditioning of Phi, so the check measures the drift the updates accumulate.
  // M' rows of the changed orbitals and the new rows Binv'[c_b], both staged [r][NeP] where
  // Bc and D were (no longer read), so the r x r dots read on-chip copies
  T* Mr = Bc;
  T* Bn = D;
  constexpr int KU = 32 / sizeof(T);
  for (int bi = warp; bi < r; bi += kCommitWarps) {
    const T* src_row = Bb + (size_t)ms.slot[bi] * Ne;
    T* dst_row = Bn + (size_t)bi * NeP;
    if (vrow) {
      for (int kv = lane; kv < Ne / V; kv += 32) {
        T v[V];
        vld(src_row + kv * V, v);
        vst(dst_row + kv * V, v);
      }
    } else {
      for (int k = lane; k < Ne; k += 32) dst_row[k] = src_row[k];
    }
  }
  for (int ai = warp; ai < r; ai += kCommitWarps) {
    const int o = ms.orb[ai], sp = o >= N ? 1 : 0;
    const T* hf = ms.feat[ms.sidx[ai]];
    for (int k0 = 0; k0 < Ne; k0 += 32 * KU) {
      T m[KU];
#pragma unroll
      for (int u = 0; u < KU; ++u) {
        const int k = k0 + lane + 32 * u;
        m[u] = k < Ne ? net.M0b[(size_t)o * Ne + k] : T(0);
      }
#pragma unroll 4
      for (int c = 0; c < h; ++c) {
        const T hc = hf[c];
        const T* wr = net.proj_w + (size_t)c * 2 * Ne + sp * Ne;
#pragma unroll
        for (int u = 0; u < KU; ++u) {
          const int k = k0 + lane + 32 * u;
          if (k < Ne) m[u] += hc * wr[k];
        }
      }
#pragma unroll
      for (int u = 0; u < KU; ++u) {
        const int k = k0 + lane + 32 * u;
        if (k < Ne) Mr[(size_t)ai * NeP + k] = m[u];
      }
    }
  }
  __syncthreads();
  // squared norms: nrm[a] = |M'_a|^2, nrm[kRMax + b] = |Binv'[c_b]|^2
  for (int q = warp; q < 2 * r; q += kCommitWarps) {
    const T* row = q < r ? Mr + (size_t)q * NeP : Bn + (size_t)(q - r) * NeP;
    T s = T(0);
    for (int k = lane; k < Ne; k += 32) s += row[k] * row[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) nrm[q < r ? q : kRMax + q - r] = s;
  }
  __syncthreads();
  T worst = T(0);
  for (int ai = warp; ai < r; ai += kCommitWarps) {
    const T* mrow = Mr + (size_t)ai * NeP;
    for (int b0 = 0; b0 < r; b0 += 4) {
      T acc[4] = {T(0), T(0), T(0), T(0)};
      for (int k = lane; k < Ne; k += 32) {
        const T mv = mrow[k];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += mv * Bn[(size_t)min(b0 + q, r - 1) * NeP + k];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
        if (b0 + q < r) {
          const T den = sqrt(nrm[ai] * nrm[kRMax + b0 + q]);
          const T res = den > T(0) ? fabs(acc[q] - (ai == b0 + q ? T(1) : T(0))) / den : T(INFINITY);
          worst = (res > worst || res != res) ? res : worst;
        }
      }
    }
  }
  if (lane == 0) {
    // non-negative doubles order like their bit patterns (NaN above +inf)
    const double w = (double)worst;
    atomicMax(&s_drift_bits, (unsigned long long)__double_as_longlong(w != w ? (double)INFINITY : w));
  }
  __syncthreads();
  if (tid == 0) {
    const double dr = __longlong_as_double((long long)s_drift_bits);
    a.drift[b] = fmax(a.drift[b], dr);
    atomicMax(a.drift_max_bits, s_drift_bits);
    if (dr > a.drift_tol) a.status[b] |= SCALE_SAMPLE_DRIFT;
  }
}

// The samples that need an FP64 re-factorisation -- all of them (force_all), a sample whose
// drift check fired or whose Woodbury step was skipped, and (when counters_due) a sample
// whose commit counter reached refresh_every -- compacted into list[0, *count); the rest
// of list is -1 (set before the launch). The order of the entries is arbitrary; every
// sample is re-factorised on its own.
__global__ void k_mark_refresh(int B, int refresh_every, bool force_all, bool counters_due,
                               const int32_t* __restrict__ commits, const int32_t* __restrict__ status,
                               int32_t* __restrict__ list, int32_t* __restrict__ count,
                               int32_t* __restrict__ n_refresh, int32_t* __restrict__ n_drift) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int st = status[b];
  const bool bad = st & (SCALE_SAMPLE_BAD_COUNT | SCALE_SAMPLE_DOUBLE_OCC);
  const bool drift = st & SCALE_SAMPLE_DRIFT;
  const bool need = !bad && (force_all || drift || (counters_due && commits[b] >= refresh_every));
  if (need) list[atomicAdd(count, 1)] = b;
  if (need) {
    atomicAdd(n_refresh, 1);
    if (drift && !force_all) atomicAdd(n_drift, 1);
  }
}

template <typename T, int H>
cudaError_t commit_t(scale_ctx* c, const int32_t* moves, const int32_t* pick, const int32_t* dir, const double* u,
                     int32_t* accepted) {
  CommitArgs a{};
  a.lat = c->lat;
  a.k0 = c->k0;
  a.occ = c->occ;
  a.slot_of_orb = c->slot_of_orb;
  a.orb_of_slot = c->orb_of_slot;
  a.z0 = c->z0;
  a.HL = c->HL;
  a.Binv = c->Binv;
  a.Pt = c->Pt;
  a.G0t = c->G0t;
  a.logabs = c->logabs;
  a.sign_slot = c->sign_slot;
  a.status = c->status;
  a.commits = c->commits;
  a.drift = c->drift;
  a.drift_tol = c->arch.drift_tol;
  a.moves = moves;
  a.scratch = c->commit_scratch;
  a.drift_max_bits = reinterpret_cast<unsigned long long*>(c->stat_dev);
  a.n_commits = reinterpret_cast<int32_t*>(c->stat_dev + 1);
  a.mf.wf = c->use_mma ? (const WFrag*)c->wfrag : nullptr;
  a.mf.kind = mma_kind_of(c->arch.precision);
  a.mf.oscale = c->use_mma && a.mf.kind == kFP16 ? fp16_scales(c) + kMaxLayers : nullptr;
  a.pick = pick;
  a.dir = dir;
  a.u = u;
  a.accepted = accepted;
  const int NeP = (c->Ne + 3) & ~3;
  // Bc and D in shared memory while two CTAs per SM still fit (both, else D alone, else none)
  constexpr size_t kLimit = 110 * 1024;
  int bc_smem = 1, d_smem = 1;
  if (commit_smem<T, H>(c->N, NeP, true, true).total > kLimit) bc_smem = 0;
  if (!bc_smem && commit_smem<T, H>(c->N, NeP, false, true).total > kLimit) d_smem = 0;
  const size_t smem = commit_smem<T, H>(c->N, NeP, bc_smem, d_smem).total;
  cudaError_t e = cudaFuncSetAttribute(k_commit<T, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_commit<T, H><<<c->B, kCommitThreads, smem, c->stream>>>(a, make_net<T>(c), bc_smem, d_smem);
  return cudaGetLastError();
}

}  // namespace

static cudaError_t commit_dispatch(scale_ctx* c, const int32_t* moves, const int32_t* pick, const int32_t* dir,
                                   const double* u, int32_t* accepted) {
  if (c->hpad == 16)
    return c->fp64 ? commit_t<double, 16>(c, moves, pick, dir, u, accepted)
                   : commit_t<float, 16>(c, moves, pick, dir, u, accepted);
  if (c->hpad == 32)
    return c->fp64 ? commit_t<double, 32>(c, moves, pick, dir, u, accepted)
                   : commit_t<float, 32>(c, moves, pick, dir, u, accepted);
  return c->fp64 ? commit_t<double, 64>(c, moves, pick, dir, u, accepted)
                 : commit_t<float, 64>(c, moves, pick, dir, u, accepted);
}

cudaError_t launch_commit(scale_ctx* c, const int32_t* moves) {
  return commit_dispatch(c, moves, nullptr, nullptr, nullptr, nullptr);
}

cudaError_t launch_metropolis(scale_ctx* c, const int32_t* pick, const int32_t* dir, const double* u,
                              int32_t* accepted) {
  return commit_dispatch(c, nullptr, pick, dir, u, accepted);
}

cudaError_t launch_mark_refresh(scale_ctx* c, bool force_all, bool counters_due) {
  int32_t* counters = reinterpret_cast<int32_t*>(c->stat_dev + 1);
  cudaError_t e = cudaMemsetAsync(c->list, 0xff, sizeof(int32_t) * (size_t)c->B, c->stream);  // all -1
  if (e == cudaSuccess) e = cudaMemsetAsync(c->list_count, 0, sizeof(int32_t), c->stream);
  if (e != cudaSuccess) return e;
  k_mark_refresh<<<(c->B + 255) / 256, 256, 0, c->stream>>>(c->B, c->arch.refresh_every, force_all, counters_due,
                                                            c->commits, c->status, c->list, c->list_count,
                                                            counters + 1, counters + 2);
  return cudaGetLastError();
}

}  // namespace scale
