// symmetry.cu -- the symmetry-projected amplitude (App. "Symmetry Projection")
//     psi_sym(n) = sum_g Pi(n, g) chi_g psi(g n)
// for the loaded samples. Each group element is an orbital permutation perm[g][o]
// (o = s*N + i): g n occupies perm[g][o] for every orbital o occupied in n, and Pi(n, g) is
// the parity of the permutation that sorts the images of n's occupied orbitals (listed in
// ascending order) -- the fermionic sign of the relabelling. Per group element the images
// g n of the whole batch are built, evaluated by the network forward and a
// determinant-only FP64 LU (the |G| evaluations per sample the projection costs), and
// added to a per-sample FP64 sum kept as s * exp(m) with the largest log|psi| first.
#include <algorithm>

#include "scale_internal.cuh"

namespace scale {

namespace {

constexpr int kThreads = 256;

// g n and Pi(n, g) of sample b (one CTA per sample). Pi counts the pairs o < o' of
// occupied orbitals whose images are out of order. An image outside the model's space
// (particle numbers other than n_up / n_dn -- which also catches two occupied orbitals sent
// to one --, a double occupancy in t-J, or an occupied orbital sent outside [0, 2N)) gets
// Pi = 0: its amplitude is zero.
__global__ void __launch_bounds__(kThreads) k_apply_group(Lattice lat, const int8_t* __restrict__ occ,
                                                          const int32_t* __restrict__ perm,
                                                          int8_t* __restrict__ occ_out, int32_t* __restrict__ pi) {
  extern __shared__ int sm[];
  const int N = lat.N;
  int* pg = sm;                                              // [2N]
  int* bits = pg + 2 * N;                                    // [N] new site states
  unsigned char* on = reinterpret_cast<unsigned char*>(bits + N);  // [2N]
  __shared__ int s_par, s_bad, s_up, s_dn;
  const int b = blockIdx.x, tid = threadIdx.x;
  const int8_t* ob = occ + (size_t)b * N;
  if (tid == 0) s_par = s_bad = s_up = s_dn = 0;
  for (int o = tid; o < 2 * N; o += kThreads) {
    pg[o] = perm[o];
    on[o] = (ob[o % N] >> (o / N)) & 1;
  }
  for (int i = tid; i < N; i += kThreads) bits[i] = 0;
  __syncthreads();
  int par = 0, bad = 0;
  for (int o = tid; o < 2 * N; o += kThreads) {
    if (!on[o]) continue;
    const int img = pg[o];
    if (img < 0 || img >= 2 * N) {
      bad = 1;
      continue;
    }
    atomicOr(&bits[img % N], 1 << (img / N));
    for (int o2 = o + 1; o2 < 2 * N; ++o2) par ^= (on[o2] && pg[o2] < img) ? 1 : 0;
  }
  if (par) atomicXor(&s_par, 1);
  if (bad) atomicOr(&s_bad, 1);
  __syncthreads();
  int nu = 0, nd = 0;
  for (int i = tid; i < N; i += kThreads) {
    const int v = bits[i];
    occ_out[(size_t)b * N + i] = (int8_t)v;
    nu += v & 1;
    nd += v >> 1;
    if (v == 3 && lat.model == SCALE_MODEL_TJ) bad = 1;
  }
  if (nu) atomicAdd(&s_up, nu);
  if (nd) atomicAdd(&s_dn, nd);
  if (bad) atomicOr(&s_bad, 1);
  __syncthreads();
  if (tid == 0) {
    const bool invalid = s_bad || s_up != lat.n_up || s_dn != lat.n_dn;
    pi[b] = invalid ? 0 : (s_par ? -1 : 1);
  }
}

__global__ void k_sym_init(int B, double* __restrict__ m, double* __restrict__ s) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) {
    m[b] = -INFINITY;
    s[b] = 0.0;
  }
}

// s * exp(m) += chi * Pi * sign(psi(g n)) * exp(log|psi(g n)|)
__global__ void k_sym_accum(int B, const double* __restrict__ chi, const double* __restrict__ la,
                            const int32_t* __restrict__ sg, const int32_t* __restrict__ pi,
                            double* __restrict__ m, double* __restrict__ s) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const double c = chi[0] * (double)pi[b] * (double)sg[b];
  if (c == 0.0) return;
  const double l = la[b];
  if (l > m[b]) {
    s[b] = s[b] * exp(m[b] - l) + c;
    m[b] = l;
  } else {
    s[b] += c * exp(l - m[b]);
  }
}

__global__ void k_sym_final(int B, const double* __restrict__ m, const double* __restrict__ s,
                            double* __restrict__ logabs, int32_t* __restrict__ sign) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const double v = s[b];
  logabs[b] = v == 0.0 ? -INFINITY : m[b] + log(fabs(v));
  sign[b] = v > 0.0 ? 1 : (v < 0.0 ? -1 : 0);
}

}  // namespace

cudaError_t launch_log_psi_sym(scale_ctx* c, int G, const int32_t* perms, const double* chi, double* logabs,
                               int32_t* sign) {
  const int B = c->B, N = c->N, nb = (B + 255) / 256;
  double* m = c->full_la;
  double* s = c->full_diag;
  int32_t* pi = c->full_sg;
  int8_t* gocc = c->full_occ;
  k_sym_init<<<nb, 256, 0, c->stream>>>(B, m, s);
  cudaError_t e = cudaGetLastError();
  const size_t smem = sizeof(int) * 3 * N + 2 * N + 16;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_apply_group, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  for (int g = 0; g < G && e == cudaSuccess; ++g) {
    k_apply_group<<<B, kThreads, smem, c->stream>>>(c->lat, c->occ, perms + (size_t)g * 2 * N, gocc, pi);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    // the images are new configurations: forward without touching the cached features,
    // then the determinant alone (FP64 LU) in ascending orbital order
    if ((e = launch_forward(c, gocc, B, nullptr, false, c->Phi64)) != cudaSuccess) break;
    if ((e = launch_gj(c, c->Phi64, c->Ne, B, nullptr, false, true, nullptr, c->la_tmp, c->sg_tmp, nullptr)) !=
        cudaSuccess)
      break;
    k_sym_accum<<<nb, 256, 0, c->stream>>>(B, chi + g, c->la_tmp, c->sg_tmp, pi, m, s);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  k_sym_final<<<nb, 256, 0, c->stream>>>(B, m, s, logabs, sign);
  return cudaGetLastError();
}

}  // namespace scale
