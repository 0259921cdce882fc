// grad.cu -- per-sample d log|psi| / d theta by a hand-written backward pass.
//
//   d log|det Phi| / d Phi[a][k] = (Phi^-1)[k][a] = Binv[a][k]   (row a = slot a)
//   proj_b[s*Ne+k]     += sum_{slots a of spin s} Binv[a][k]
//   proj_w[c][s*Ne+k]  += sum_{slots a of spin s} H(L)_{i_a}[c] Binv[a][k]
//   dH(L)_i[c]          = sum_{s: (s,i) occupied} Pt[s][slot(s,i)][c]     (Pt = W_s Binv)
//   layer l (out = res*in + act(z), z = b + sum_d K[d]^T in_{i+d}, d over the stencil's taps:
//   the k x k box, or its offsets within L2 distance (k-1)/2, weights stored per tap):
//     dz = dout * act'(z); db = sum_i dz_i; dK[d][ci][co] = sum_i in_{i+d}[ci] dz_i[co]
//     din_j = res*dout_j + sum_d K[d] dz_{j-d}
//   embedding row E_i[n_i] += dH(0)_i.
// The forward is recomputed from the current occupations (all layers stored, or, with
// recompute = 1, only every ceil(sqrt(L))-th layer input, the rest recomputed per segment).
#include <algorithm>
#include <cmath>

#include "scale_internal.cuh"

namespace scale {

namespace {

// Forward layer writing explicit output / pre-activation slabs ([B][N][h] each).
template <typename T>
__global__ void k_fwd_layer(Lattice lat, Net<T> net, int l, const int8_t* __restrict__ occ, const T* __restrict__ in,
                            T* __restrict__ out, T* __restrict__ zout) {
  const int h = net.h, N = lat.N;
  const int b = blockIdx.y;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * h) return;
  const int i = idx / h, c = idx - i * h;
  const int k = net.ksize[l], r = (k - 1) / 2;
  const int8_t* ob = occ + (size_t)b * N;
  T z = net.bias[l][c];
  int d = 0;  // tap index, row-major over the box
  for (int ky = 0; ky < k; ++ky)
    for (int kx = 0; kx < k; ++kx) {
      if (!stencil_in(net.stencil, k, kx - r, ky - r)) continue;
      const int t = d++;
      const int j = site_off(lat, i, kx - r, ky - r);
      if (j < 0) continue;
      const T* w = net.kernel[l] + (size_t)t * h * h + c;
      const T* x = (l == 0) ? net.embed + ((size_t)(net.per_site ? j * 4 : 0) + (ob[j] & 3)) * h
                            : in + ((size_t)b * N + j) * h;
      for (int ci = 0; ci < h; ++ci) z += x[ci] * w[(size_t)ci * h];
    }
  T self = T(0);
  if (net.resid[l])
    self = (l == 0) ? net.embed[((size_t)(net.per_site ? i * 4 : 0) + (ob[i] & 3)) * h + c] : in[((size_t)b * N + i) * h + c];
  out[(size_t)b * N * h + idx] = self + act_fn<T>(net.act, z);
  zout[(size_t)b * N * h + idx] = z;
}

// Projection gradients and dH(L).
template <typename T>
__global__ void k_grad_proj(Lattice lat, Net<T> net, const int32_t* __restrict__ orb_of_slot,
                            const int32_t* __restrict__ slot_of_orb, const T* __restrict__ Binv,
                            const T* __restrict__ Pt, const T* __restrict__ HLr, int64_t off_pw, int64_t off_pb,
                            int64_t P, double* __restrict__ grad, T* __restrict__ dH) {
  const int b = blockIdx.x;
  const int N = lat.N, Ne = lat.Ne, h = net.h;
  const T* Bb = Binv + (size_t)b * Ne * Ne;
  const T* Hb = HLr + (size_t)b * N * h;
  double* g = grad + (size_t)b * P;
  const int32_t* os = orb_of_slot + (size_t)b * Ne;
  for (int q = threadIdx.x; q < 2 * Ne * (h + 1); q += blockDim.x) {
    const int s = q / (Ne * (h + 1));
    const int rem = q - s * Ne * (h + 1);
    const int c = rem / Ne, k = rem - c * Ne;  // c == h: bias
    double acc = 0.0;
    for (int a = 0; a < Ne; ++a) {
      const int o = os[a];
      if (o / N != s) continue;
      const int i = o - s * N;
      const double bv = (double)Bb[(size_t)a * Ne + k];
      acc += (c == h) ? bv : (double)Hb[(size_t)i * h + c] * bv;
    }
    if (c == h)
      g[off_pb + s * Ne + k] = acc;
    else
      g[off_pw + (size_t)c * 2 * Ne + s * Ne + k] = acc;
  }
  const int32_t* so = slot_of_orb + (size_t)b * 2 * N;
  const T* Pb = Pt + (size_t)b * 2 * Ne * h;
  for (int q = threadIdx.x; q < N * h; q += blockDim.x) {
    const int i = q / h, c = q - i * h;
    T acc = T(0);
    for (int s = 0; s < 2; ++s) {
      const int a = so[s * N + i];
      if (a >= 0) acc += Pb[((size_t)s * Ne + a) * h + c];
    }
    dH[(size_t)b * N * h + q] = acc;
  }
}

// dz = dout * act'(z), and the bias gradient.
template <typename T>
__global__ void k_grad_dz(Lattice lat, Net<T> net, int l, const T* __restrict__ dout, const T* __restrict__ z,
                          T* __restrict__ dz, int64_t off_b, int64_t P, double* __restrict__ grad) {
  const int b = blockIdx.x;
  const int N = lat.N, h = net.h;
  for (int q = threadIdx.x; q < N * h; q += blockDim.x)
    dz[(size_t)b * N * h + q] = dout[(size_t)b * N * h + q] * act_grad<T>(net.act, z[(size_t)b * N * h + q]);
  __syncthreads();
  for (int c = threadIdx.x; c < h; c += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < N; ++i) acc += (double)dz[((size_t)b * N + i) * h + c];
    grad[(size_t)b * P + off_b + c] = acc;
  }
}

// dK[d][ci][co] = sum_i in_{i+d}[ci] dz_i[co], accumulated in the mode's precision (FP32 in
// mixed precision: an FP64 sum would run on GB300's few FP64 units for no accuracy the FP32
// activations carry)
template <typename T>
__global__ void k_grad_kernel(Lattice lat, Net<T> net, int l, int taps, const int8_t* __restrict__ occ,
                              const T* __restrict__ in, const T* __restrict__ dz, int64_t off_k, int64_t P,
                              double* __restrict__ grad) {
  const int b = blockIdx.y;
  const int N = lat.N, h = net.h, k = net.ksize[l];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= taps * h * h) return;
  const int d = q / (h * h), rem = q - d * h * h, ci = rem / h, co = rem - ci * h;
  int dx, dy;
  stencil_tap(net.stencil, k, d, dx, dy);
  const int8_t* ob = occ + (size_t)b * N;
  T acc = T(0);
  for (int i = 0; i < N; ++i) {
    const int j = site_off(lat, i, dx, dy);
    if (j < 0) continue;
    const T xin = (l == 0) ? net.embed[((size_t)(net.per_site ? j * 4 : 0) + (ob[j] & 3)) * h + ci]
                           : in[((size_t)b * N + j) * h + ci];
    acc += xin * dz[((size_t)b * N + i) * h + co];
  }
  grad[(size_t)b * P + off_k + q] = (double)acc;
}

// KT[d][co][ci] = K[d][ci][co] of one layer (the loads of k_grad_din are then consecutive
// across the lanes of a warp).
template <typename T>
__global__ void k_transpose_taps(const T* __restrict__ K, int taps, int h, T* __restrict__ KT) {
  const int total = taps * h * h;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const int d = q / (h * h), rem = q - d * h * h, ci = rem / h, co = rem - ci * h;
    KT[(size_t)d * h * h + (size_t)co * h + ci] = K[q];
  }
}

// din_j[ci] = res*dout_j[ci] + sum_d sum_co K[d][ci][co] dz_{j-d}[co]; KT = the layer's
// kernel transposed per tap ([d][co][ci]).
template <typename T>
__global__ void k_grad_din(Lattice lat, Net<T> net, int l, const T* __restrict__ KT, const T* __restrict__ dout,
                           const T* __restrict__ dz, T* __restrict__ din) {
  const int b = blockIdx.y;
  const int N = lat.N, h = net.h, k = net.ksize[l], r = (k - 1) / 2;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N * h) return;
  const int j = q / h, ci = q - j * h;
  T acc = net.resid[l] ? dout[(size_t)b * N * h + q] : T(0);
  int d = 0;  // tap index, row-major over the box
  for (int ky = 0; ky < k; ++ky)
    for (int kx = 0; kx < k; ++kx) {
      if (!stencil_in(net.stencil, k, kx - r, ky - r)) continue;
      const int t = d++;
      const int i = site_off(lat, j, -(kx - r), -(ky - r));  // site i with i + d = j
      if (i < 0) continue;
      const T* w = KT + (size_t)t * h * h + ci;
      const T* g = dz + ((size_t)b * N + i) * h;
      for (int co = 0; co < h; ++co) acc += w[(size_t)co * h] * g[co];
    }
  din[(size_t)b * N * h + q] = acc;
}

// Embedding rows: E_i[n_i] (per-site tables) or E[n] summed over sites (shared table).
template <typename T>
__global__ void k_grad_embed(Lattice lat, Net<T> net, const int8_t* __restrict__ occ, const T* __restrict__ dH0,
                             int64_t P, double* __restrict__ grad) {
  const int b = blockIdx.x;
  const int N = lat.N, h = net.h;
  const int8_t* ob = occ + (size_t)b * N;
  double* g = grad + (size_t)b * P;
  if (net.per_site) {
    for (int q = threadIdx.x; q < N * h; q += blockDim.x) {
      const int i = q / h, c = q - i * h;
      g[((size_t)i * 4 + (ob[i] & 3)) * h + c] = (double)dH0[(size_t)b * N * h + q];
    }
  } else {
    for (int q = threadIdx.x; q < 4 * h; q += blockDim.x) {
      const int n = q / h, c = q - n * h;
      double acc = 0.0;
      for (int i = 0; i < N; ++i)
        if (ob[i] == n) acc += (double)dH0[((size_t)b * N + i) * h + c];
      g[q] = acc;
    }
  }
}

__global__ void k_nan_bad(int B, int64_t P, const int32_t* __restrict__ status, double* __restrict__ grad) {
  const int b = blockIdx.x;
  if (!(status[b] & (SCALE_SAMPLE_BAD_COUNT | SCALE_SAMPLE_DOUBLE_OCC | SCALE_SAMPLE_SINGULAR))) return;
  for (int64_t q = threadIdx.x; q < P; q += blockDim.x) grad[(size_t)b * P + q] = CUDART_NAN;
}

template <typename T>
cudaError_t grad_t(scale_ctx* c, double* grad, int recompute) {
  const Net<T> net = make_net<T>(c);
  const int B = c->B, N = c->N, h = c->h, L = c->L;
  const size_t slab = (size_t)B * N * h;  // elements of one layer slab
  const int stride = recompute ? std::max(1, (int)std::ceil(std::sqrt((double)L))) : 1;
  // slabs: checkpoints (layer inputs 1..L-1 at multiples of stride), segment H and z
  // (stride + 1 and stride), dH ping-pong (2), dz (1)
  const int n_ck = (L + stride - 1) / stride;
  size_t ktaps = 0;  // transposed kernels of every layer
  for (int l = 0; l < L; ++l) ktaps += (size_t)stencil_taps(net.stencil, net.ksize[l]) * h * h;
  const size_t need = sizeof(T) * (slab * (size_t)(n_ck + (stride + 1) + stride + 3) + ktaps);
  if (need > c->grad_scratch_bytes) {
    if (c->grad_scratch) cudaFree(c->grad_scratch);
    c->grad_scratch = nullptr;
    c->grad_scratch_bytes = 0;
    cudaError_t e = cudaMalloc(&c->grad_scratch, need);
    if (e != cudaSuccess) return e;
    c->grad_scratch_bytes = need;
  }
  T* base = (T*)c->grad_scratch;
  T* ck = base;                                 // [n_ck] slabs: input of layer m*stride
  T* segH = ck + (size_t)n_ck * slab;           // [stride+1]
  T* segZ = segH + (size_t)(stride + 1) * slab; // [stride]
  T* dA = segZ + (size_t)stride * slab;
  T* dB = dA + slab;
  T* dZ = dB + slab;
  T* KT = dZ + slab;  // [sum over layers of taps * h * h]
  cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(double) * (size_t)B * c->P, c->stream);
  if (e != cudaSuccess) return e;
  T* KTl[kMaxLayers];
  {
    size_t o = 0;
    for (int l = 0; l < L; ++l) {
      const int tl = stencil_taps(net.stencil, net.ksize[l]);
      KTl[l] = KT + o;
      k_transpose_taps<T><<<(tl * h * h + 255) / 256, 256, 0, c->stream>>>(net.kernel[l], tl, h, KTl[l]);
      o += (size_t)tl * h * h;
    }
  }
  // offsets
  int64_t off = (int64_t)(c->arch.per_site_embed ? N : 1) * 4 * h;
  int64_t offK[kMaxLayers], offB[kMaxLayers];
  int taps[kMaxLayers];
  for (int l = 0; l < L; ++l) {
    taps[l] = stencil_taps(net.stencil, net.ksize[l]);
    offK[l] = off;
    off += (int64_t)taps[l] * h * h;
    offB[l] = off;
    off += h;
  }
  const int64_t off_pw = off, off_pb = off + (int64_t)h * 2 * c->Ne;
  dim3 gridL((N * h + 127) / 128, B);
  // forward pass storing the checkpoints; H(L) of the recomputed forward lands in dA
  // temporarily (the projection gradient reads it)
  {
    const T* in = nullptr;
    for (int l = 0; l < L; ++l) {
      T* out = (l + 1) % stride == 0 && (l + 1) / stride < n_ck ? ck + (size_t)((l + 1) / stride) * slab
                                                               : segH + (size_t)((l + 1) % 2) * slab;
      if (l == L - 1) out = dB;
      k_fwd_layer<T><<<gridL, 128, 0, c->stream>>>(c->lat, net, l, c->occ, in, out, segZ);
      in = out;
    }
  }
  k_grad_proj<T><<<B, 256, 0, c->stream>>>(c->lat, net, c->orb_of_slot, c->slot_of_orb, (const T*)c->Binv,
                                           (const T*)c->Pt, dB, off_pw, off_pb, c->P, grad, dA);
  T* dcur = dA;   // d/dH(l+1)
  T* dnext = dB;  // d/dH(l)
  for (int seg = n_ck - 1; seg >= 0; --seg) {
    const int l0 = seg * stride, l1 = std::min(L, l0 + stride);
    // recompute the segment forward from its checkpoint: segH[m] = H(l0+m), segZ[m] = z(l0+m)
    const T* in = (l0 == 0) ? nullptr : ck + (size_t)seg * slab;
    for (int l = l0; l < l1; ++l) {
      T* out = segH + (size_t)(l - l0 + 1) * slab;
      k_fwd_layer<T><<<gridL, 128, 0, c->stream>>>(c->lat, net, l, c->occ, in, out, segZ + (size_t)(l - l0) * slab);
      in = out;
    }
    for (int l = l1 - 1; l >= l0; --l) {
      const T* lin = (l == 0) ? nullptr : (l == l0 ? ck + (size_t)seg * slab : segH + (size_t)(l - l0) * slab);
      k_grad_dz<T><<<B, 256, 0, c->stream>>>(c->lat, net, l, dcur, segZ + (size_t)(l - l0) * slab, dZ, offB[l], c->P,
                                             grad);
      const int kq = taps[l] * h * h;
      k_grad_kernel<T><<<dim3((kq + 127) / 128, B), 128, 0, c->stream>>>(c->lat, net, l, taps[l], c->occ, lin, dZ,
                                                                          offK[l], c->P, grad);
      k_grad_din<T><<<gridL, 128, 0, c->stream>>>(c->lat, net, l, KTl[l], dcur, dZ, dnext);
      std::swap(dcur, dnext);
    }
  }
  k_grad_embed<T><<<B, 256, 0, c->stream>>>(c->lat, net, c->occ, dcur, c->P, grad);
  k_nan_bad<<<B, 256, 0, c->stream>>>(B, c->P, c->status, grad);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_grad(scale_ctx* c, double* grad, int recompute) {
  return c->fp64 ? grad_t<double>(c, grad, recompute) : grad_t<float>(c, grad, recompute);
}

}  // namespace scale
