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
  double* logabs;
  int32_t* sign_slot;
  int32_t* status;
  int32_t* commits;
  double* drift;
  double drift_tol;
  const int32_t* moves;
  void* scratch;          // [B][3*kRMax*Ne + 2*kRMax*kMaxH] T : X, D, saved Binv rows, saved Pt rows
  unsigned long long* drift_max_bits;
  int32_t* n_commits;
  MlpFrags mf;
};

// In-place inverse of the r x r matrix R (warp; lane j owns column j), Gauss-Jordan with
// partial pivoting and explicit row swaps. Returns the determinant.
template <typename T>
__device__ T warp_inverse(T (*R)[kRMax + 1], T (*Ri)[kRMax + 1], int r) {
  const int lane = threadIdx.x & 31;
  if (lane < r)
    for (int i = 0; i < r; ++i) Ri[i][lane] = (i == lane) ? T(1) : T(0);
  __syncwarp();
  T det = T(1);
  for (int k = 0; k < r; ++k) {
    int p = k;
    if (lane == k) {
      T best = fabs(R[k][k]);
      for (int i = k + 1; i < r; ++i)
        if (fabs(R[i][k]) > best) {
          best = fabs(R[i][k]);
          p = i;
        }
    }
    p = __shfl_sync(0xffffffffu, p, k);
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
    const T inv = T(1) / pv;
    // scale the pivot row, eliminate column k from every other row
    T rk = T(0), rik = T(0);
    if (lane < r) {
      rk = R[k][lane] * inv;
      rik = Ri[k][lane] * inv;
    }
    __syncwarp();
    if (lane < r) {
      R[k][lane] = rk;
      Ri[k][lane] = rik;
    }
    __syncwarp();
    for (int i = 0; i < r; ++i) {
      if (i == k) continue;
      const T f = R[i][k];
      __syncwarp();
      if (lane < r) {
        R[i][lane] -= f * rk;
        Ri[i][lane] -= f * rik;
      }
      __syncwarp();
    }
  }
  return det;
}

template <typename T, int H>
__global__ void __launch_bounds__(256) k_commit(CommitArgs a, Net<T> net) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = a.lat.N, Ne = a.lat.Ne, h = net.h;
  MoveScratch<T, H>& ms = *reinterpret_cast<MoveScratch<T, H>*>(smem);
  T(*z0n)[H] = reinterpret_cast<T(*)[H]>(&ms + 1);   // [kSMax][H]
  T(*Ri)[kRMax + 1] = reinterpret_cast<T(*)[kRMax + 1]>(z0n + kSMax);
  int32_t* slot_s = reinterpret_cast<int32_t*>(Ri + kRMax);
  int8_t* occ_s = reinterpret_cast<int8_t*>(slot_s + 2 * N);
  __shared__ int s_go;
  __shared__ double s_det;
  __shared__ double s_drift;

  const int b = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int32_t* mv = a.moves + (size_t)b * 4;
  const int kind = mv[0], src = mv[1], dst = mv[2], spin = mv[3];
  const int st = a.status[b];
  if (kind < 0 || (st & (SCALE_SAMPLE_BAD_COUNT | SCALE_SAMPLE_DOUBLE_OCC | SCALE_SAMPLE_SINGULAR))) return;
  for (int i = tid; i < N; i += blockDim.x) occ_s[i] = a.occ[(size_t)b * N + i];
  for (int o = tid; o < 2 * N; o += blockDim.x) slot_s[o] = a.slot_of_orb[(size_t)b * 2 * N + o];
  __syncthreads();
  if (!move_allowed(a.lat, kind, src, dst, spin, occ_s)) return;  // uniform across the CTA

  T* zb = (T*)a.z0 + (size_t)b * N * h;
  T* hb = (T*)a.HL + (size_t)b * N * h;
  T* Bb = (T*)a.Binv + (size_t)b * Ne * Ne;
  T* Pb = (T*)a.Pt + (size_t)b * 2 * Ne * h;
  T* X = (T*)a.scratch + (size_t)b * (3 * kRMax * Ne + 2 * kRMax * kMaxH);
  T* D = X + (size_t)kRMax * Ne;
  T* Bc = D + (size_t)kRMax * Ne;
  T* Pc = Bc + (size_t)kRMax * Ne;  // [2][r][h]

  SampleView<T> sv;
  sv.occ = occ_s;
  sv.slot_of_orb = slot_s;
  sv.z0 = zb;
  sv.HL = hb;
  sv.Binv = Bb;
  sv.Pt = Pb;
  if (warp == 0) {
    if (lane == 0) {
      ms.kind = kind;
      ms.src = src;
      ms.dst = dst;
      ms.spin = spin;
    }
    __syncwarp();
    move_features<T, H>(a.lat, net, a.k0, sv, a.mf, ms, z0n);
    const int r = move_matrix<T, H>(a.lat, net, sv, ms);
    T det = T(0);
    if (r > 0) det = warp_inverse<T>(ms.R, Ri, r);
    if (lane == 0) {
      s_go = (r > 0 && det != T(0)) ? 1 : 0;
      s_det = (double)det;
    }
  }
  __syncthreads();
  if (!s_go) return;
  const int r = ms.r;
  // X[a][j] = Phi'_C Phi^-1 - E_C^T: moved rows take G(o'_a, j), every row the
  // Delta H_{s_a} . Pt[s_a][j] term, and -1 at j = c_a for the moved rows only (the
  // identity of an unmoved row cancels against E_C^T).
  for (int q = tid; q < r * Ne; q += blockDim.x) {
    const int ai = q / Ne, j = q - ai * Ne;
    const int o = ms.orb[ai], sp = o / N, i = o - sp * N;
    const T* pt = Pb + ((size_t)sp * Ne + j) * h;
    T v = T(0);
    if (ms.moved[ai]) {
      // G(o', j) with the new features: (M0[o'] + proj_b) . Binv[j] + H'_i . Pt[j]
      const T* fnew = ms.feat[ms.sidx[ai]];
      const T* brow = Bb + (size_t)j * Ne;
      const T* m0b = net.M0b + (size_t)o * Ne;
      for (int k = 0; k < Ne; ++k) v += m0b[k] * brow[k];
      for (int c = 0; c < h; ++c) v += fnew[c] * pt[c];
      if (j == ms.slot[ai]) v -= T(1);
    } else {
      const T* dh = ms.hl[ms.sidx[ai]];  // Delta H (move_matrix left it there)
      for (int c = 0; c < h; ++c) v += dh[c] * pt[c];
    }
    (void)i;
    X[(size_t)ai * Ne + j] = v;
  }
  __syncthreads();
  // D = R^-1 X; save the rows Binv[c_b] and Pt[s][c_b] before they change
  for (int q = tid; q < r * Ne; q += blockDim.x) {
    const int bi = q / Ne, j = q - bi * Ne;
    T v = T(0);
    for (int ai = 0; ai < r; ++ai) v += Ri[bi][ai] * X[(size_t)ai * Ne + j];
    D[(size_t)bi * Ne + j] = v;
    Bc[(size_t)bi * Ne + j] = Bb[(size_t)ms.slot[bi] * Ne + j];
  }
  __syncthreads();
  for (int q = tid; q < 2 * r * h; q += blockDim.x) {
    const int sp = q / (r * h), rem = q - sp * r * h, bi = rem / h, c = rem - bi * h;
    Pc[q] = Pb[((size_t)sp * Ne + ms.slot[bi]) * h + c];
  }
  __syncthreads();
  // Binv[j][k] -= sum_b D[b][j] Bc[b][k]
  for (int q = tid; q < Ne * Ne; q += blockDim.x) {
    const int j = q / Ne, k = q - j * Ne;
    T acc = Bb[q];
    for (int bi = 0; bi < r; ++bi) acc -= D[(size_t)bi * Ne + j] * Bc[(size_t)bi * Ne + k];
    Bb[q] = acc;
  }
  // Pt[s][j][c] -= sum_b D[b][j] Pc[s][b][c]
  for (int q = tid; q < 2 * Ne * h; q += blockDim.x) {
    const int sp = q / (Ne * h), rem = q - sp * Ne * h, j = rem / h, c = rem - j * h;
    T acc = Pb[q];
    for (int bi = 0; bi < r; ++bi) acc -= D[(size_t)bi * Ne + j] * Pc[((size_t)sp * r + bi) * h + c];
    Pb[q] = acc;
  }
  // features on S: z0 <- z0', H(L) <- H'(L)
  for (int q = tid; q < ms.nS * h; q += blockDim.x) {
    const int s = q / h, c = q - s * h;
    const int site = ms.site[s];
    zb[(size_t)site * h + c] = z0n[s][c];
    hb[(size_t)site * h + c] = ms.feat[s][c];
  }
  __syncthreads();
  if (tid == 0) {
    // occupations and slot maps: moved electrons keep their rows
    const int n_src = occ_s[src], n_dst = occ_s[dst];
    if (kind == 0) {
      const int slot = slot_s[spin * N + src];
      a.slot_of_orb[(size_t)b * 2 * N + spin * N + src] = -1;
      a.slot_of_orb[(size_t)b * 2 * N + spin * N + dst] = slot;
      a.orb_of_slot[(size_t)b * Ne + slot] = spin * N + dst;
    } else {
      const int s_up = (n_src == 1) ? 0 : 1;  // spin on src before the exchange
      const int s_dn = 1 - s_up;               // spin on dst before the exchange
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
    s_drift = 0.0;
  }
  __syncthreads();
  // Drift check on the changed rows, accumulated in FP64: the normalised residual
  //   max_{a,b} | M'[o'_a] . Binv'[c_b] - delta_ab | / (|M'[o'_a]|_2 |Binv'[c_b]|_2),
  // M'[o'] = M0[o'] + proj_b[s] + H'(L)_i W_s with the updated features (rows built once).
  // Normalised this way a freshly rounded inverse sits near the working precision whatever
  // the conditioning of Phi, so the check measures the drift the updates accumulate.
  T* Mr = X;  // [r][Ne]
  for (int q = tid; q < r * Ne; q += blockDim.x) {
    const int ai = q / Ne, k = q - ai * Ne;
    const int o = ms.orb[ai], sp = o / N, i = o - sp * N;
    const T* hrow = hb + (size_t)i * h;
    T m = net.M0b[(size_t)o * Ne + k];
    for (int c = 0; c < h; ++c) m += hrow[c] * net.proj_w[(size_t)c * 2 * Ne + sp * Ne + k];
    Mr[q] = m;
  }
  __syncthreads();
  double worst = 0.0;
  for (int q = tid; q < r * r; q += blockDim.x) {
    const int ai = q / r, bi = q - ai * r;
    const T* brow = Bb + (size_t)ms.slot[bi] * Ne;
    const T* mrow = Mr + (size_t)ai * Ne;
    double acc = 0.0, nm = 0.0, nb = 0.0;
    for (int k = 0; k < Ne; ++k) {
      acc += (double)mrow[k] * (double)brow[k];
      nm += (double)mrow[k] * (double)mrow[k];
      nb += (double)brow[k] * (double)brow[k];
    }
    const double den = sqrt(nm * nb);
    worst = fmax(worst, den > 0.0 ? fabs(acc - (ai == bi ? 1.0 : 0.0)) / den : INFINITY);
  }
  for (int off = 16; off > 0; off >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, off));
  if (lane == 0) {
    // positive doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long*>(&s_drift), (unsigned long long)__double_as_longlong(worst));
  }
  __syncthreads();
  if (tid == 0) {
    a.drift[b] = fmax(a.drift[b], s_drift);
    atomicMax(a.drift_max_bits, (unsigned long long)__double_as_longlong(s_drift));
    if (s_drift > a.drift_tol) a.status[b] |= SCALE_SAMPLE_DRIFT;
  }
}

// list[b] = b when sample b needs an FP64 re-factorisation, else -1.
__global__ void k_mark_refresh(int B, int refresh_every, bool force_all, const int32_t* __restrict__ commits,
                               const int32_t* __restrict__ status, int32_t* __restrict__ list,
                               int32_t* __restrict__ n_refresh, int32_t* __restrict__ n_drift) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int st = status[b];
  const bool bad = st & (SCALE_SAMPLE_BAD_COUNT | SCALE_SAMPLE_DOUBLE_OCC);
  const bool drift = st & SCALE_SAMPLE_DRIFT;
  const bool need = !bad && (force_all || drift || commits[b] >= refresh_every);
  list[b] = need ? b : -1;
  if (need) {
    atomicAdd(n_refresh, 1);
    if (drift && !force_all) atomicAdd(n_drift, 1);
  }
}

template <typename T, int H>
cudaError_t commit_t(scale_ctx* c, const int32_t* moves) {
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
  a.mf.kind = c->arch.precision == SCALE_PREC_MIXED_BF16 ? kBF16 : kTF32;
  const size_t smem = sizeof(MoveScratch<T, H>) + sizeof(T) * kSMax * H + sizeof(T) * kRMax * (kRMax + 1) +
                      sizeof(int32_t) * 2 * c->N + c->N + 16;
  cudaError_t e = cudaFuncSetAttribute(k_commit<T, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_commit<T, H><<<c->B, 256, smem, c->stream>>>(a, make_net<T>(c));
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_commit(scale_ctx* c, const int32_t* moves) {
  if (c->hpad == 16) return c->fp64 ? commit_t<double, 16>(c, moves) : commit_t<float, 16>(c, moves);
  if (c->hpad == 32) return c->fp64 ? commit_t<double, 32>(c, moves) : commit_t<float, 32>(c, moves);
  return c->fp64 ? commit_t<double, 64>(c, moves) : commit_t<float, 64>(c, moves);
}

cudaError_t launch_mark_refresh(scale_ctx* c, bool force_all) {
  int32_t* counters = reinterpret_cast<int32_t*>(c->stat_dev + 1);
  k_mark_refresh<<<(c->B + 255) / 256, 256, 0, c->stream>>>(c->B, c->arch.refresh_every, force_all, c->commits,
                                                            c->status, c->list, counters + 1, counters + 2);
  return cudaGetLastError();
}

}  // namespace scale
