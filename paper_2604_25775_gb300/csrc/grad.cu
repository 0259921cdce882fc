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

// Four consecutive elements through the read-only path (16-byte aligned: h % 4 == 0 and
// every slab, table and weight block starts on a multiple of four elements).
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 q = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = q.x;
  v[1] = q.y;
  v[2] = q.z;
  v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p)), c = __ldg(reinterpret_cast<const double2*>(p) + 1);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = c.x;
  v[3] = c.y;
}

// Input row of site j for layer l: the embedding row E_j[n_j] for layer 0, else the slab row.
template <typename T>
__device__ __forceinline__ const T* layer_in_row(const Net<T>& net, int l, const int8_t* ob, const T* in_b, int j,
                                                 int h) {
  return l == 0 ? net.embed + ((size_t)(net.per_site ? j * 4 : 0) + (ob[j] & 3)) * h : in_b + (size_t)j * h;
}

// Forward layer (h % 4 == 0), 4 sites x 4 output channels per thread, the same summation order
// as k_fwd_layer (bias, taps in row-major order, input channels ascending).
template <typename T, int HC>
__global__ void k_fwd_tile(Lattice lat, Net<T> net, int l, const int8_t* __restrict__ occ, const T* __restrict__ in,
                           T* __restrict__ out, T* __restrict__ zout) {
  const int h = HC ? HC : net.h, N = lat.N, hq = h >> 2;
  const int b = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ((N + 3) >> 2) * hq) return;
  const int sq = q / hq, c0 = (q - sq * hq) * 4;
  const int k = net.ksize[l], r = (k - 1) / 2;
  const int8_t* ob = occ + (size_t)b * N;
  const T* in_b = in + (size_t)b * N * h;  // unused for layer 0
  T acc[4][4];
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int m = 0; m < 4; ++m) acc[s][m] = net.bias[l][c0 + m];
  int d = 0;
  for (int ky = 0; ky < k; ++ky)
    for (int kx = 0; kx < k; ++kx) {
      if (!stencil_in(net.stencil, k, kx - r, ky - r)) continue;
      const int t = d++;
      const T* row[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int i = sq * 4 + s;
        const int j = i < N ? site_off(lat, i, kx - r, ky - r) : -1;
        row[s] = j < 0 ? nullptr : layer_in_row(net, l, ob, in_b, j, h);
      }
      const T* w = net.kernel[l] + (size_t)t * h * h + c0;
#pragma unroll
      for (int ci = 0; ci < h; ci += 4) {
        T wv[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a) ld4(w + (size_t)(ci + a) * h, wv[a]);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          if (!row[s]) continue;
          T xv[4];
          ld4(row[s] + ci, xv);
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int m = 0; m < 4; ++m) acc[s][m] = fma(xv[a], wv[a][m], acc[s][m]);
        }
      }
    }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int i = sq * 4 + s;
    if (i >= N) break;
    const size_t o = ((size_t)b * N + i) * h + c0;
    const T* self = net.resid[l] ? layer_in_row(net, l, ob, in_b, i, h) + c0 : nullptr;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      out[o + m] = (self ? self[m] : T(0)) + act_fn<T>(net.act, acc[s][m]);
      zout[o + m] = acc[s][m];
    }
  }
}

// dK[d][ci][co] = sum_i in_{i+d}[ci] dz_i[co] (h % 8 == 0): one thread per (tap, 4 input
// channels, 8 output channels), sites in ascending order as in k_grad_kernel.
template <typename T, int HC>
__global__ void k_dk_tile(Lattice lat, Net<T> net, int l, int taps, const int8_t* __restrict__ occ,
                          const T* __restrict__ in, const T* __restrict__ dz, int64_t off_k, int64_t P,
                          double* __restrict__ grad) {
  const int b = blockIdx.y;
  const int N = lat.N, h = HC ? HC : net.h, hq = h >> 2, ho = h >> 3, k = net.ksize[l];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= taps * hq * ho) return;
  const int t = q / (hq * ho), rem = q - t * hq * ho, ci0 = (rem / ho) * 4, co0 = (rem % ho) * 8;
  int dx, dy;
  stencil_tap(net.stencil, k, t, dx, dy);
  const int8_t* ob = occ + (size_t)b * N;
  const T* in_b = in + (size_t)b * N * h;
  const T* dz_b = dz + (size_t)b * N * h + co0;
  T acc[4][8] = {};
  for (int y = 0; y < lat.Ly; ++y) {  // every branch below is uniform over a warp (same tap, site)
    int yy = y + dy;
    if (yy < 0 || yy >= lat.Ly) {
      if (!lat.pbc_y) continue;
      yy = ((yy % lat.Ly) + lat.Ly) % lat.Ly;
    }
#pragma unroll 2
    for (int x = 0; x < lat.Lx; ++x) {
      int xx = x + dx;
      if (xx < 0 || xx >= lat.Lx) {
        if (!lat.pbc_x) continue;
        xx = ((xx % lat.Lx) + lat.Lx) % lat.Lx;
      }
      T xv[4], gv[2][4];
      ld4(layer_in_row(net, l, ob, in_b, yy * lat.Lx + xx, h) + ci0, xv);
      const T* gr = dz_b + (size_t)(y * lat.Lx + x) * h;
      ld4(gr, gv[0]);
      ld4(gr + 4, gv[1]);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[a][m] = fma(xv[a], gv[m >> 2][m & 3], acc[a][m]);
    }
  }
  double* g = grad + (size_t)b * P + off_k + (size_t)t * h * h + co0;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int m = 0; m < 8; ++m) g[(size_t)(ci0 + a) * h + m] = (double)acc[a][m];
}

// din_j[ci] = res*dout_j[ci] + sum_d sum_co K[d][ci][co] dz_{j-d}[co] (h % 4 == 0), 4 sites x
// 4 input channels per thread; KT = the layer's kernel transposed per tap ([d][co][ci]).
template <typename T, int HC>
__global__ void k_din_tile(Lattice lat, Net<T> net, int l, const T* __restrict__ KT, const T* __restrict__ dout,
                           const T* __restrict__ dz, T* __restrict__ din) {
  const int h = HC ? HC : net.h, N = lat.N, hq = h >> 2;
  const int b = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ((N + 3) >> 2) * hq) return;
  const int sq = q / hq, c0 = (q - sq * hq) * 4;
  const int k = net.ksize[l], r = (k - 1) / 2;
  const size_t base = (size_t)b * N * h;
  T acc[4][4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int j = sq * 4 + s;
#pragma unroll
    for (int m = 0; m < 4; ++m) acc[s][m] = (net.resid[l] && j < N) ? dout[base + (size_t)j * h + c0 + m] : T(0);
  }
  int d = 0;
  for (int ky = 0; ky < k; ++ky)
    for (int kx = 0; kx < k; ++kx) {
      if (!stencil_in(net.stencil, k, kx - r, ky - r)) continue;
      const int t = d++;
      const T* g[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int j = sq * 4 + s;
        const int i = j < N ? site_off(lat, j, -(kx - r), -(ky - r)) : -1;  // site i with i + d = j
        g[s] = i < 0 ? nullptr : dz + base + (size_t)i * h;
      }
      const T* w = KT + (size_t)t * h * h + c0;
#pragma unroll
      for (int co = 0; co < h; co += 4) {
        T wv[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a) ld4(w + (size_t)(co + a) * h, wv[a]);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          if (!g[s]) continue;
          T gv[4];
          ld4(g[s] + co, gv);
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int m = 0; m < 4; ++m) acc[s][m] = fma(wv[a][m], gv[a], acc[s][m]);
        }
      }
    }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int j = sq * 4 + s;
    if (j >= N) break;
#pragma unroll
    for (int m = 0; m < 4; ++m) din[base + (size_t)j * h + c0 + m] = acc[s][m];
  }
}

// ---- the forward and dK with one sample's slabs staged in shared memory --------------------
// CTA per sample: the layer input rows (the embedding rows for layer 0) and, for dK, dz copied
// to shared memory once with coalesced loads, and the site table nbr[i][t] (the site reached
// from i by tap t; -1 past an open edge). The register tiles and the summation order are those
// of the kernels above, so the results are the same.
__device__ __forceinline__ void lds4(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x;
  v[1] = q.y;
  v[2] = q.z;
  v[3] = q.w;
}
__device__ __forceinline__ void lds4(const double* p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p), c = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = c.x;
  v[3] = c.y;
}

__device__ __forceinline__ void stage_nbr(const Lattice& lat, int stencil, int k, int taps, int sgn, int* nbr) {
  for (int q = threadIdx.x; q < lat.N * taps; q += blockDim.x) {
    const int i = q / taps, t = q - i * taps;
    int dx, dy;
    stencil_tap(stencil, k, t, dx, dy);
    nbr[q] = site_off(lat, i, sgn * dx, sgn * dy);
  }
}

// Bytes of shared memory of the staged kernels: [slabs][N][h] rows and the [N][taps] table.
inline size_t grad_smem_bytes(int N, int h, int taps, int slabs, size_t tsize) {
  return (size_t)slabs * N * h * tsize + (size_t)N * taps * sizeof(int);
}

template <typename T, int HC>
__global__ void k_fwd_smem(Lattice lat, Net<T> net, int l, int taps, const int8_t* __restrict__ occ,
                           const T* __restrict__ in, T* __restrict__ out, T* __restrict__ zout) {
  extern __shared__ __align__(16) unsigned char gsm[];
  const int h = HC ? HC : net.h, N = lat.N, hq = h >> 2;
  const int b = blockIdx.x;
  T* xs = reinterpret_cast<T*>(gsm);
  int* nbr = reinterpret_cast<int*>(xs + (size_t)N * h);
  const int8_t* ob = occ + (size_t)b * N;
  const T* in_b = in + (size_t)b * N * h;
  for (int q = threadIdx.x; q < N * h; q += blockDim.x) {
    const int i = q / h, c = q - i * h;
    xs[q] = layer_in_row(net, l, ob, in_b, i, h)[c];
  }
  stage_nbr(lat, net.stencil, net.ksize[l], taps, 1, nbr);
  __syncthreads();
  const int tiles = ((N + 3) >> 2) * hq;
  for (int q = threadIdx.x; q < tiles; q += blockDim.x) {
    const int sq = q / hq, c0 = (q - sq * hq) * 4;
    T acc[4][4];
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int m = 0; m < 4; ++m) acc[s][m] = net.bias[l][c0 + m];
    for (int t = 0; t < taps; ++t) {
      int row[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int i = sq * 4 + s;
        row[s] = i < N ? nbr[i * taps + t] : -1;
      }
      const T* w = net.kernel[l] + (size_t)t * h * h + c0;
#pragma unroll
      for (int ci = 0; ci < h; ci += 4) {
        T wv[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a) ld4(w + (size_t)(ci + a) * h, wv[a]);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          if (row[s] < 0) continue;
          T xv[4];
          lds4(xs + (size_t)row[s] * h + ci, xv);
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int m = 0; m < 4; ++m) acc[s][m] = fma(xv[a], wv[a][m], acc[s][m]);
        }
      }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int i = sq * 4 + s;
      if (i >= N) break;
      const size_t o = ((size_t)b * N + i) * h + c0;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        out[o + m] = (net.resid[l] ? xs[(size_t)i * h + c0 + m] : T(0)) + act_fn<T>(net.act, acc[s][m]);
        zout[o + m] = acc[s][m];
      }
    }
  }
}

template <typename T, int HC>
__global__ void k_dk_smem(Lattice lat, Net<T> net, int l, int taps, const int8_t* __restrict__ occ,
                          const T* __restrict__ in, const T* __restrict__ dz, int64_t off_k, int64_t P,
                          double* __restrict__ grad) {
  extern __shared__ __align__(16) unsigned char gsm[];
  const int N = lat.N, h = HC ? HC : net.h, hq = h >> 2, ho = h >> 3;
  const int b = blockIdx.x;
  T* xs = reinterpret_cast<T*>(gsm);
  T* gs = xs + (size_t)N * h;
  int* nbr = reinterpret_cast<int*>(gs + (size_t)N * h);
  const int8_t* ob = occ + (size_t)b * N;
  const T* in_b = in + (size_t)b * N * h;
  const T* dz_b = dz + (size_t)b * N * h;
  for (int q = threadIdx.x; q < N * h; q += blockDim.x) {
    const int i = q / h, c = q - i * h;
    xs[q] = layer_in_row(net, l, ob, in_b, i, h)[c];
    gs[q] = dz_b[q];
  }
  stage_nbr(lat, net.stencil, net.ksize[l], taps, 1, nbr);
  __syncthreads();
  for (int q = threadIdx.x; q < taps * hq * ho; q += blockDim.x) {
    const int t = q / (hq * ho), rem = q - t * hq * ho, ci0 = (rem / ho) * 4, co0 = (rem % ho) * 8;
    T acc[4][8] = {};
    for (int i = 0; i < N; ++i) {
      const int j = nbr[i * taps + t];
      if (j < 0) continue;
      T xv[4], gv[2][4];
      lds4(xs + (size_t)j * h + ci0, xv);
      lds4(gs + (size_t)i * h + co0, gv[0]);
      lds4(gs + (size_t)i * h + co0 + 4, gv[1]);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int m = 0; m < 8; ++m) acc[a][m] = fma(xv[a], gv[m >> 2][m & 3], acc[a][m]);
    }
    double* g = grad + (size_t)b * P + off_k + (size_t)t * h * h + co0;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int m = 0; m < 8; ++m) g[(size_t)(ci0 + a) * h + m] = (double)acc[a][m];
  }
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
    T acc = T(0);  // the mode's precision, as the layer gradients
    for (int a = 0; a < Ne; ++a) {
      const int i = os[a] - s * N;
      if (i < 0 || i >= N) continue;  // a slot of the other spin
      const T bv = Bb[(size_t)a * Ne + k];
      acc += (c == h) ? bv : Hb[(size_t)i * h + c] * bv;
    }
    if (c == h)
      g[off_pb + s * Ne + k] = (double)acc;
    else
      g[off_pw + (size_t)c * 2 * Ne + s * Ne + k] = (double)acc;
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
  if (net.per_site) {  // every row written: the three rows of a site's other states get 0
    for (int q = threadIdx.x; q < N * 4 * h; q += blockDim.x) {
      const int i = q / (4 * h), rem = q - i * 4 * h, n = rem / h, c = rem - n * h;
      g[q] = n == (ob[i] & 3) ? (double)dH0[((size_t)b * N + i) * h + c] : 0.0;
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

// One CTA per sample with `smem` bytes of staged slabs; the block covers the sample's work
// (one tile per thread up to 1024 tiles, beyond that each thread loops over its share).
template <typename... KA, typename... A>
cudaError_t staged_launch(void (*kern)(KA...), int B, int work, size_t smem, cudaStream_t st, A... args) {
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int block = std::min(1024, std::max(32, (work + 31) / 32 * 32));  // one tile per thread
  kern<<<B, block, smem, st>>>(args...);
  return cudaGetLastError();
}

constexpr size_t kGradSmemMax = 96 * 1024;  // staged slabs up to this size (a few CTAs per SM)

template <typename T>
cudaError_t grad_t(scale_ctx* c, double* grad, int recompute) {
  const Net<T> net = make_net<T>(c);
  const int B = c->B, N = c->N, h = c->h, L = c->L;
  const size_t slab = (size_t)B * N * h;  // elements of one layer slab
  const bool tiled = h % 8 == 0;          // the register-tiled kernels (vector loads of 4)
  int max_taps = 1;
  for (int l = 0; l < L; ++l) max_taps = std::max(max_taps, stencil_taps(net.stencil, net.ksize[l]));
  // the tiled kernels with one sample's slabs staged in shared memory: small lattices (the
  // 16x4 cylinder: forward 109 -> 96 us, dK 216 -> 140 us per 2048 walkers); at 256 sites the
  // 73 KB of staged slabs per sample cost more than the L1-served kernels (measured)
  const bool staged = tiled && N <= 128 && grad_smem_bytes(N, h, max_taps, 2, sizeof(T)) <= kGradSmemMax;
  // stored: every layer's input and pre-activation kept from the one forward pass; recompute:
  // only every stride-th layer input, each segment's forward recomputed during the backward
  const int stride = recompute ? std::max(1, (int)std::ceil(std::sqrt((double)L))) : 1;
  const int n_ck = (L + stride - 1) / stride;
  // slabs: checkpoints (layer inputs at multiples of stride), segment H and z (stored: all L
  // pre-activations, no segment H), H(L), dH ping-pong (2), dz (1)
  const size_t n_seg = recompute ? (size_t)(stride + 1) + stride : (size_t)L;
  size_t ktaps = 0;  // transposed kernels of every layer
  for (int l = 0; l < L; ++l) ktaps += (size_t)stencil_taps(net.stencil, net.ksize[l]) * h * h;
  const size_t need = sizeof(T) * (slab * (n_ck + n_seg + 4) + ktaps);
  if (need > c->grad_scratch_bytes) {
    if (c->grad_scratch) cudaFree(c->grad_scratch);
    c->grad_scratch = nullptr;
    c->grad_scratch_bytes = 0;
    cudaError_t e = cudaMalloc(&c->grad_scratch, need);
    if (e != cudaSuccess) return e;
    c->grad_scratch_bytes = need;
  }
  T* base = (T*)c->grad_scratch;
  T* ck = base;                          // [n_ck] slabs: input of layer m*stride (slab 0 unused)
  T* seg = ck + (size_t)n_ck * slab;     // recompute: segH [stride+1], segZ [stride]; stored: Z [L]
  T* segH = seg;
  T* segZ = recompute ? seg + (size_t)(stride + 1) * slab : seg;
  T* HL = seg + n_seg * slab;
  T* dA = HL + slab;
  T* dB = dA + slab;
  T* dZ = dB + slab;
  T* KT = dZ + slab;  // [sum over layers of taps * h * h]
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
  // offsets (every parameter is written below: no clearing pass over the B x P gradients)
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
  const dim3 gridL((N * h + 127) / 128, B), gridT((((N + 3) / 4) * (h / 4) + 127) / 128, B);
  // the tiled kernels with the width as a compile-time constant where it is a common one
#define SCALE_GRAD_TILED(KERNEL, GRID, ...)                                                \
  switch (h) {                                                                             \
    case 8: KERNEL<T, 8><<<GRID, 128, 0, c->stream>>>(__VA_ARGS__); break;                 \
    case 16: KERNEL<T, 16><<<GRID, 128, 0, c->stream>>>(__VA_ARGS__); break;               \
    case 32: KERNEL<T, 32><<<GRID, 128, 0, c->stream>>>(__VA_ARGS__); break;               \
    case 64: KERNEL<T, 64><<<GRID, 128, 0, c->stream>>>(__VA_ARGS__); break;               \
    default: KERNEL<T, 0><<<GRID, 128, 0, c->stream>>>(__VA_ARGS__);                       \
  }
#define SCALE_GRAD_STAGED(KERNEL, WORK, SMEM, ...)                                                            \
  switch (h) {                                                                                               \
    case 8: e = staged_launch(KERNEL<T, 8>, B, WORK, SMEM, c->stream, __VA_ARGS__); break;                   \
    case 16: e = staged_launch(KERNEL<T, 16>, B, WORK, SMEM, c->stream, __VA_ARGS__); break;                 \
    case 32: e = staged_launch(KERNEL<T, 32>, B, WORK, SMEM, c->stream, __VA_ARGS__); break;                 \
    case 64: e = staged_launch(KERNEL<T, 64>, B, WORK, SMEM, c->stream, __VA_ARGS__); break;                 \
    default: e = staged_launch(KERNEL<T, 0>, B, WORK, SMEM, c->stream, __VA_ARGS__);                         \
  }
  const int site_tiles = ((N + 3) / 4) * (h / 4);
  cudaError_t e = cudaSuccess;
  auto fwd = [&](int l, const T* in, T* out, T* z) {
    if (staged) {
      const int tl = stencil_taps(net.stencil, net.ksize[l]);
      SCALE_GRAD_STAGED(k_fwd_smem, site_tiles, grad_smem_bytes(N, h, tl, 1, sizeof(T)), c->lat, net, l, tl, c->occ,
                        in, out, z);
    } else if (tiled) {
      SCALE_GRAD_TILED(k_fwd_tile, gridT, c->lat, net, l, c->occ, in, out, z);
    } else {
      k_fwd_layer<T><<<gridL, 128, 0, c->stream>>>(c->lat, net, l, c->occ, in, out, z);
    }
  };
  // forward pass: layer inputs at the checkpoints (every layer when stored), H(L) last
  {
    const T* in = nullptr;
    for (int l = 0; l < L; ++l) {
      T* out = HL;
      if (l < L - 1) {
        const bool keep = (l + 1) % stride == 0;
        out = keep ? ck + (size_t)((l + 1) / stride) * slab : segH + (size_t)((l + 1) % 2) * slab;
      }
      fwd(l, in, out, recompute ? segZ : segZ + (size_t)l * slab);
      if (e != cudaSuccess) return e;
      in = out;
    }
  }
  k_grad_proj<T><<<B, 256, 0, c->stream>>>(c->lat, net, c->orb_of_slot, c->slot_of_orb, (const T*)c->Binv,
                                           (const T*)c->Pt, HL, off_pw, off_pb, c->P, grad, dA);
  T* dcur = dA;   // d/dH(l+1)
  T* dnext = dB;  // d/dH(l)
  for (int sg = n_ck - 1; sg >= 0; --sg) {
    const int l0 = sg * stride, l1 = std::min(L, l0 + stride);
    if (recompute) {  // segment forward from its checkpoint: segH[m] = H(l0+m), segZ[m] = z(l0+m)
      const T* in = (l0 == 0) ? nullptr : ck + (size_t)sg * slab;
      for (int l = l0; l < l1; ++l) {
        T* out = segH + (size_t)(l - l0 + 1) * slab;
        fwd(l, in, out, segZ + (size_t)(l - l0) * slab);
        if (e != cudaSuccess) return e;
        in = out;
      }
    }
    for (int l = l1 - 1; l >= l0; --l) {
      const T* lin = (l == 0) ? nullptr : (l == l0 ? ck + (size_t)sg * slab : segH + (size_t)(l - l0) * slab);
      const T* zl = recompute ? segZ + (size_t)(l - l0) * slab : segZ + (size_t)l * slab;
      k_grad_dz<T><<<B, 256, 0, c->stream>>>(c->lat, net, l, dcur, zl, dZ, offB[l], c->P, grad);
      const int kq = tiled ? taps[l] * (h / 4) * (h / 8) : taps[l] * h * h;
      if (staged) {
        SCALE_GRAD_STAGED(k_dk_smem, kq, grad_smem_bytes(N, h, taps[l], 2, sizeof(T)), c->lat, net, l, taps[l], c->occ,
                          lin, dZ, offK[l], c->P, grad);
        if (e != cudaSuccess) return e;
        // the input gradient reads dz through L1 as fast as from a staged copy (measured)
        SCALE_GRAD_TILED(k_din_tile, gridT, c->lat, net, l, KTl[l], dcur, dZ, dnext);
      } else if (tiled) {
        const dim3 gridK((kq + 127) / 128, B);
        SCALE_GRAD_TILED(k_dk_tile, gridK, c->lat, net, l, taps[l], c->occ, lin, dZ, offK[l], c->P, grad);
        SCALE_GRAD_TILED(k_din_tile, gridT, c->lat, net, l, KTl[l], dcur, dZ, dnext);
      } else {
        k_grad_kernel<T><<<dim3((kq + 127) / 128, B), 128, 0, c->stream>>>(c->lat, net, l, taps[l], c->occ, lin,
                                                                            dZ, offK[l], c->P, grad);
        k_grad_din<T><<<gridL, 128, 0, c->stream>>>(c->lat, net, l, KTl[l], dcur, dZ, dnext);
      }
      std::swap(dcur, dnext);
    }
  }
#undef SCALE_GRAD_TILED
#undef SCALE_GRAD_STAGED
  k_grad_embed<T><<<B, 256, 0, c->stream>>>(c->lat, net, c->occ, dcur, c->P, grad);
  k_nan_bad<<<B, 256, 0, c->stream>>>(B, c->P, c->status, grad);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_grad(scale_ctx* c, double* grad, int recompute) {
  return c->fp64 ? grad_t<double>(c, grad, recompute) : grad_t<float>(c, grad, recompute);
}

}  // namespace scale
