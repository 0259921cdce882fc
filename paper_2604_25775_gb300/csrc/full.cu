// full.cu -- the full-recompute comparison path (Sec. III.A): psi(n) and every connected
// amplitude psi(n') by a fresh network forward and a fresh LU of the Slater matrix, the
// O(N^4) route that the low-rank update replaces. Same enumeration order as the low-rank
// path. Nothing cached by the context enters the result: psi(n) is recomputed alongside its
// connected configurations.
//
// Matrix elements here are in the ascending-orbital convention, with the Jordan-Wigner
// signs explicit:
//   hop      c+_{dst,s} c_{src,s}:  -t (-1)^(occupied orbitals strictly between)
//   exchange (J/2) S+_i S-_j = -(J/2)(c+_{i up} c_{j up})(c+_{j dn} c_{i dn}):
//            -(J/2) (-1)^(k_up + k_dn), k_s = occupied spin-s orbitals strictly between.
//
// Precision: the network and the Slater matrix in the mode's precision (as at load), every
// determinant by the FP64 LU with partial pivoting. An FP32 LU of a 224 x 224 Slater matrix
// would carry cond(Phi) x 2^-24 relative error in each amplitude, far above the mixed-mode
// tolerance on the ill-conditioned matrices of random configurations.
//
// Scheduling: every call is asynchronous. Sample b owns count[b] + 1 entries (entry 0 is n
// itself, entry m >= 1 its (m-1)-th connected configuration); a device-side exclusive scan
// gives their global offsets, and the host walks the entries in fixed-size chunks up to the
// capacity B * (max_moves + 1). Chunk positions past the device-side total are marked -1 in
// the chunk's list, and every kernel of the chunk skips them, so the host never reads a count.
#include <algorithm>

#include "scale_internal.cuh"

namespace scale {

namespace {

__device__ int between_count(const int8_t* occ, int N, int o1, int o2) {
  const int lo = min(o1, o2), hi = max(o1, o2);
  int cnt = 0;
  for (int o = lo + 1; o < hi; ++o) {
    const int s = o / N, i = o - s * N;
    cnt += (occ[i] >> s) & 1;
  }
  return cnt;
}

// Enumerate the connected configurations of every sample: moves [B][cap][4], ascending
// convention coefficients [B][cap], count [B], diagonal [B].
__global__ void k_enum(Lattice lat, const int8_t* __restrict__ occ, const int32_t* __restrict__ bonds, int nb_nn,
                       int nb_nnn, const int32_t* __restrict__ status, int cap, int32_t* __restrict__ moves,
                       double* __restrict__ coeff, int32_t* __restrict__ count, double* __restrict__ diag) {
  const int b = blockIdx.x;
  if (threadIdx.x != 0) return;
  const int N = lat.N;
  const int8_t* x = occ + (size_t)b * N;
  int n = 0;
  if (status[b] & (SCALE_SAMPLE_BAD_COUNT | SCALE_SAMPLE_DOUBLE_OCC | SCALE_SAMPLE_SINGULAR)) {
    count[b] = 0;
    diag[b] = CUDART_NAN;
    return;
  }
  double d = 0.0;
  if (lat.model == SCALE_MODEL_HUBBARD) {
    int nd = 0;
    for (int i = 0; i < N; ++i) nd += x[i] == 3;
    d = lat.U * nd;
  } else if (lat.model == SCALE_MODEL_HUBBARD_PH) {
    int nu = 0;  // U sum_i n_up (1 - n_dn)
    for (int i = 0; i < N; ++i) nu += x[i] == 1;
    d = lat.U * nu;
  } else {
    for (int q = 0; q < nb_nn; ++q) {
      const int i = bonds[2 * q], j = bonds[2 * q + 1];
      d += lat.J * 0.5 * ((x[i] & 1) - ((x[i] >> 1) & 1)) * 0.5 * ((x[j] & 1) - ((x[j] >> 1) & 1));
    }
  }
  diag[b] = d;
  const int nb = nb_nn + nb_nnn;
  for (int q = 0; q < nb; ++q)
    for (int s = 0; s < 2; ++s) {
      const int i = bonds[2 * q], j = bonds[2 * q + 1];
      const bool hi = (x[i] >> s) & 1, hj = (x[j] >> s) & 1;
      if (hi == hj) continue;
      const int src = hi ? i : j, dst = hi ? j : i;
      if (lat.model == SCALE_MODEL_TJ && x[dst] != 0) continue;
      if (n < cap) {
        int32_t* m = moves + ((size_t)b * cap + n) * 4;
        m[0] = 0; m[1] = src; m[2] = dst; m[3] = s;
        const double t = (q < nb_nn) ? lat.t : lat.tp;
        const int k = between_count(x, N, s * N + src, s * N + dst);
        coeff[(size_t)b * cap + n] = -t * ((k & 1) ? -1.0 : 1.0);
      }
      ++n;
    }
  if (lat.model == SCALE_MODEL_TJ && lat.J != 0.0)
    for (int q = 0; q < nb_nn; ++q) {
      const int i = bonds[2 * q], j = bonds[2 * q + 1];
      if (!((x[i] == 1 && x[j] == 2) || (x[i] == 2 && x[j] == 1))) continue;
      if (n < cap) {
        int32_t* m = moves + ((size_t)b * cap + n) * 4;
        m[0] = 1; m[1] = i; m[2] = j; m[3] = 0;
        const int k = between_count(x, N, i, j) + between_count(x, N, N + i, N + j);
        coeff[(size_t)b * cap + n] = -0.5 * lat.J * ((k & 1) ? -1.0 : 1.0);
      }
      ++n;
    }
  count[b] = min(n, cap);
}

// offsets[b] = sum_{b' < b} (count[b'] + extra), offsets[B] = the total (extra = 1 here: entry 0
// of a sample is n itself): one CTA, each thread scans a contiguous run of samples, then a
// scan over the threads' sums.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) k_offsets(int B, const int32_t* __restrict__ count, int extra,
                                                          int64_t* __restrict__ offsets) {
  __shared__ int64_t part[kScanThreads + 1];
  const int tid = threadIdx.x;
  const int per = (B + kScanThreads - 1) / kScanThreads;
  const int b0 = min(B, tid * per), b1 = min(B, b0 + per);
  int64_t s = 0;
  for (int b = b0; b < b1; ++b) s += (int64_t)count[b] + extra;
  part[tid] = s;
  __syncthreads();
  // Hillis-Steele inclusive scan over the 1024 partial sums
  for (int off = 1; off < kScanThreads; off <<= 1) {
    const int64_t v = tid >= off ? part[tid - off] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  int64_t run = part[tid] - s;  // exclusive prefix of this thread's run
  for (int b = b0; b < b1; ++b) {
    offsets[b] = run;
    run += (int64_t)count[b] + extra;
  }
  if (tid == kScanThreads - 1) offsets[B] = part[tid];
}

// Chunk entries [g0, g0 + G): the owning sample by binary search over the offsets, its
// configuration (entry 0: n itself; entry m: n with move m-1 applied) packed into xp[g],
// owner[g] = b * (cap + 1) + m and list[g] = g; positions past the total get list[g] = -1.
// *vcount = the number of valid positions (a prefix of the chunk).
__global__ void k_build_xprime(int N, int B, int cap, const int8_t* __restrict__ occ,
                               const int32_t* __restrict__ moves, const int64_t* __restrict__ offsets, int64_t g0,
                               int G, int8_t* __restrict__ xp, int32_t* __restrict__ owner,
                               int32_t* __restrict__ list, int32_t* __restrict__ vcount) {
  const int g = blockIdx.x;
  if (g >= G) return;
  if (g == 0 && threadIdx.x == 0) *vcount = (int32_t)max((int64_t)0, min((int64_t)G, offsets[B] - g0));
  const int64_t gg = g0 + g;
  if (gg >= offsets[B]) {
    if (threadIdx.x == 0) {
      list[g] = -1;
      owner[g] = -1;
    }
    return;
  }
  int lo = 0, hi = B;  // offsets[lo] <= gg < offsets[lo+1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if (offsets[mid] <= gg) lo = mid; else hi = mid;
  }
  const int b = lo;
  const int m = (int)(gg - offsets[b]);
  const int8_t* x = occ + (size_t)b * N;
  int8_t* y = xp + (size_t)g * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) y[i] = x[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    if (m > 0) {
      const int32_t* mv = moves + ((size_t)b * cap + (m - 1)) * 4;
      const int src = mv[1], dst = mv[2], s = mv[3];
      if (mv[0] == 0) {
        y[src] = (int8_t)(x[src] & ~(1 << s));
        y[dst] = (int8_t)(x[dst] | (1 << s));
      } else {
        y[src] = x[dst];
        y[dst] = x[src];
      }
    }
    owner[g] = b * (cap + 1) + m;
    list[g] = g;
  }
}

// Scatter the chunk's determinants to their entries: la_all / sg_all [B][cap + 1].
__global__ void k_scatter_dets(int G, const int32_t* __restrict__ owner, const double* __restrict__ la,
                               const int32_t* __restrict__ sg, double* __restrict__ la_all,
                               int32_t* __restrict__ sg_all) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  const int idx = owner[g];
  if (idx < 0) return;
  la_all[idx] = la[g];
  sg_all[idx] = sg[g];
}

// E_loc[b] = diag + sum_m coeff[m] psi(n'_m)/psi(n), fixed order; psi(n) = 0 gives NaN.
__global__ void k_reduce_terms(int B, int cap, const int32_t* __restrict__ count, const double* __restrict__ diag,
                               const double* __restrict__ coeff, const double* __restrict__ la_all,
                               const int32_t* __restrict__ sg_all, double* __restrict__ eloc) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const size_t base = (size_t)b * (cap + 1);
  const int n = count[b];
  double e = diag[b];
  if (isnan(e)) {  // invalid sample (status): no entries were evaluated
    eloc[b] = e;
    return;
  }
  const double la0 = la_all[base];
  const int sg0 = sg_all[base];
  if (sg0 == 0) {
    eloc[b] = CUDART_NAN;
    return;
  }
  for (int m = 0; m < n; ++m) {
    const int sg = sg_all[base + 1 + m];
    if (sg != 0) e += coeff[(size_t)b * cap + m] * (double)(sg * sg0) * exp(la_all[base + 1 + m] - la0);
  }
  eloc[b] = e;
}

}  // namespace

cudaError_t launch_eloc_full(scale_ctx* c, double* eloc) {
  cudaError_t e;
  const int B = c->B, cap = c->max_moves, N = c->N, Ne = c->Ne;
  k_enum<<<B, 32, 0, c->stream>>>(c->lat, c->occ, c->bonds, c->nb_nn, c->nb_nnn, c->status, cap, c->full_moves,
                                  c->full_coeff, c->move_count, c->full_diag);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_offsets<<<1, kScanThreads, 0, c->stream>>>(B, c->move_count, 1, c->full_offsets);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t bound = (int64_t)B * (cap + 1);  // the device-side total is at most this
  const int chunk = c->full_chunk;
  for (int64_t g0 = 0; g0 < bound; g0 += chunk) {
    const int G = (int)std::min<int64_t>(chunk, bound - g0);
    k_build_xprime<<<G, 128, 0, c->stream>>>(N, B, cap, c->occ, c->full_moves, c->full_offsets, g0, G, c->full_occ,
                                            c->full_owner, c->full_list, c->full_vcount);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_forward_phi(c, c->full_occ, G, c->full_list, c->full_vcount, c->Phi64)) != cudaSuccess) return e;
    if ((e = launch_gj(c, c->Phi64, Ne, G, c->full_list, false, true, nullptr, c->full_la, c->full_sg, nullptr)) !=
        cudaSuccess)
      return e;
    k_scatter_dets<<<(G + 255) / 256, 256, 0, c->stream>>>(G, c->full_owner, c->full_la, c->full_sg, c->full_la_all,
                                                           c->full_sg_all);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_reduce_terms<<<(B + 255) / 256, 256, 0, c->stream>>>(B, cap, c->move_count, c->full_diag, c->full_coeff,
                                                         c->full_la_all, c->full_sg_all, eloc);
  return cudaGetLastError();
}

cudaError_t launch_offsets(scale_ctx* c, int B, const int32_t* count, int extra, int64_t* offsets) {
  k_offsets<<<1, kScanThreads, 0, c->stream>>>(B, count, extra, offsets);
  return cudaGetLastError();
}

}  // namespace scale
