// full.cu -- the full-recompute comparison path (Sec. III.A): every connected amplitude
// psi(n') by a fresh network forward and a fresh LU of Phi(n'), the O(N^4) route that the
// low-rank update replaces. Same enumeration order as the low-rank path.
//
// Matrix elements here are in the ascending-orbital convention, with the Jordan-Wigner
// signs explicit:
//   hop      c+_{dst,s} c_{src,s}:  -t (-1)^(occupied orbitals strictly between)
//   exchange (J/2) S+_i S-_j = -(J/2)(c+_{i up} c_{j up})(c+_{j dn} c_{i dn}):
//            -(J/2) (-1)^(k_up + k_dn), k_s = occupied spin-s orbitals strictly between.
#include <algorithm>
#include <vector>

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

// Packed configurations n' for global indices [g0, g0 + G): owner sample by binary search
// over the offsets.
__global__ void k_build_xprime(int N, int B, int cap, const int8_t* __restrict__ occ,
                               const int32_t* __restrict__ moves, const int64_t* __restrict__ offsets, int64_t g0,
                               int G, int8_t* __restrict__ xp, int32_t* __restrict__ owner) {
  const int g = blockIdx.x;
  if (g >= G) return;
  const int64_t gg = g0 + g;
  int lo = 0, hi = B;  // offsets[lo] <= gg < offsets[lo+1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if (offsets[mid] <= gg) lo = mid; else hi = mid;
  }
  const int b = lo;
  const int m = (int)(gg - offsets[b]);
  const int32_t* mv = moves + ((size_t)b * cap + m) * 4;
  const int8_t* x = occ + (size_t)b * N;
  int8_t* y = xp + (size_t)g * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) y[i] = x[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    const int src = mv[1], dst = mv[2], s = mv[3];
    if (mv[0] == 0) {
      y[src] = (int8_t)(x[src] & ~(1 << s));
      y[dst] = (int8_t)(x[dst] | (1 << s));
    } else {
      y[src] = x[dst];
      y[dst] = x[src];
    }
    owner[g] = b * cap + m;
  }
}

// term[b][m] = coeff * psi(n')/psi(n) from the two log-determinants.
__global__ void k_terms(int G, int cap, const int32_t* __restrict__ owner, const double* __restrict__ coeff,
                        const double* __restrict__ la_x, const int32_t* __restrict__ sg_x,
                        const double* __restrict__ la_p, const int32_t* __restrict__ sg_p,
                        double* __restrict__ terms) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  const int idx = owner[g];
  const int b = idx / cap;
  double v = 0.0;
  if (sg_p[g] != 0 && sg_x[b] != 0) v = coeff[idx] * (double)(sg_p[g] * sg_x[b]) * exp(la_p[g] - la_x[b]);
  terms[idx] = v;
}

__global__ void k_reduce_terms(int B, int cap, const int32_t* __restrict__ count, const double* __restrict__ diag,
                               const double* __restrict__ terms, double* __restrict__ eloc) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double e = diag[b];
  for (int m = 0; m < count[b]; ++m) e += terms[(size_t)b * cap + m];
  eloc[b] = e;
}

}  // namespace

cudaError_t launch_eloc_full(scale_ctx* c, double* eloc) {
  cudaError_t e;
  const int B = c->B, cap = c->max_moves, N = c->N, Ne = c->Ne;
  k_enum<<<B, 32, 0, c->stream>>>(c->lat, c->occ, c->bonds, c->nb_nn, c->nb_nnn, c->status, cap, c->full_moves,
                                  c->full_coeff, c->move_count, c->full_diag);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // log|psi(n)| and sign in the ascending convention
  if ((e = launch_logpsi_out(c, c->la_tmp, c->sg_tmp)) != cudaSuccess) return e;
  std::vector<int32_t> cnt(B);
  if ((e = cudaMemcpyAsync(cnt.data(), c->move_count, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, c->stream)) !=
      cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
  std::vector<int64_t> off(B + 1, 0);
  for (int b = 0; b < B; ++b) off[b + 1] = off[b] + cnt[b];
  if ((e = cudaMemcpyAsync(c->full_offsets, off.data(), sizeof(int64_t) * (B + 1), cudaMemcpyHostToDevice,
                           c->stream)) != cudaSuccess)
    return e;
  const int64_t total = off[B];
  const int chunk = c->full_chunk;
  for (int64_t g0 = 0; g0 < total; g0 += chunk) {
    const int G = (int)std::min<int64_t>(chunk, total - g0);
    k_build_xprime<<<G, 128, 0, c->stream>>>(N, B, cap, c->occ, c->full_moves, c->full_offsets, g0, G, c->full_occ,
                                            c->full_owner);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_forward_phi(c, c->full_occ, G, c->Phi64)) != cudaSuccess) return e;
    if (c->fp64 || c->ace)  // ACE: FP64 determinants in both modes
      e = launch_gj(c, c->Phi64, Ne, G, nullptr, false, true, nullptr, c->full_la, c->full_sg, nullptr);
    else
      e = launch_det_f32(c, reinterpret_cast<float*>(c->Phi64), Ne, G, c->full_la, c->full_sg);
    if (e != cudaSuccess) return e;
    k_terms<<<(G + 255) / 256, 256, 0, c->stream>>>(G, cap, c->full_owner, c->full_coeff, c->la_tmp, c->sg_tmp,
                                                    c->full_la, c->full_sg, c->full_terms);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_reduce_terms<<<(B + 255) / 256, 256, 0, c->stream>>>(B, cap, c->move_count, c->full_diag, c->full_terms, eloc);
  return cudaGetLastError();
}

}  // namespace scale
