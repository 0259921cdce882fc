// forward.cu -- network forward (Sec. II.B), slot bookkeeping, Slater-matrix build,
// layer-0 conv-of-embedding table and the log|psi| output convention.
#include <algorithm>

#include "mlp_mma.cuh"
#include "scale_internal.cuh"

namespace scale {

namespace {

// One network layer for every (sample, site, channel):
//   out_i[c] = res * in_i[c] + act(b[c] + sum_{offsets d} sum_c' in_{i+d}[c'] K[d][c'][c])
// Layer 0 reads its input from the embedding tables E_i[n_i] (Sec. II.B). Offsets wrap on
// periodic axes and read zeros past open edges (Eq. conv, "same boundary conditions as
// the Hamiltonian").
template <typename T>
__global__ void k_layer(Lattice lat, Net<T> net, int l, const int8_t* __restrict__ occ,
                        const int32_t* __restrict__ list, const T* __restrict__ in, T* __restrict__ out,
                        T* __restrict__ zout, int B, const int32_t* __restrict__ count) {
  const int h = net.h, N = lat.N;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * h) return;
  const int i = idx / h, c = idx - i * h;
  const int k = net.ksize[l], r = (k - 1) / 2;
  const T* K = net.kernel[l];
  // positions in the launch: all B, or the first *count entries of a compacted list
  const int nrows = count ? min(*count, B) : B;
  for (int row = blockIdx.y; row < nrows; row += gridDim.y) {
  const int b = list ? list[row] : row;
  if (b < 0) continue;
  T z = net.bias[l][c];
  const int8_t* ob = occ + (size_t)b * N;
  const T* ib = in ? in + (size_t)b * N * h : nullptr;
  int tap = 0;
  for (int ky = 0; ky < k; ++ky)
    for (int kx = 0; kx < k; ++kx) {
      if (!stencil_in(net.stencil, k, kx - r, ky - r)) continue;
      const int tp = tap++;
      const int j = site_off(lat, i, kx - r, ky - r);
      if (j < 0) continue;
      const T* w = K + (size_t)tp * h * h + c;
      const T* x = (l == 0) ? net.embed + ((size_t)(net.per_site ? j * 4 : 0) + (ob[j] & 3)) * h
                            : ib + (size_t)j * h;
#pragma unroll 8
      for (int ci = 0; ci < h; ++ci) z += x[ci] * w[(size_t)ci * h];
    }
  T self = T(0);
  if (net.resid[l]) {
    self = (l == 0) ? net.embed[((size_t)(net.per_site ? i * 4 : 0) + (ob[i] & 3)) * h + c]
                    : ib[(size_t)i * h + c];
  }
  out[(size_t)b * N * h + idx] = self + act_fn<T>(net.act, z);
  if (zout) zout[(size_t)b * N * h + idx] = z;
  }
}

// Block-wide exclusive scan of 0/1 flags over 2N orbitals; writes the ascending list of
// occupied orbitals. Returns the count (valid in every thread).
__device__ int occupied_list(const int8_t* ob, int N, int* list_out, int* s_tmp) {
  // s_tmp: at least blockDim.x ints
  const int tid = threadIdx.x, nt = blockDim.x;
  const int per = (2 * N + nt - 1) / nt;
  const int o0 = tid * per;
  int cnt = 0;
  for (int o = o0; o < min(o0 + per, 2 * N); ++o) {
    const int s = o / N, i = o - s * N;
    cnt += (ob[i] >> s) & 1;
  }
  s_tmp[tid] = cnt;
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int t = 0; t < nt; ++t) {
      const int v = s_tmp[t];
      s_tmp[t] = acc;
      acc += v;
    }
    s_tmp[nt] = acc;
  }
  __syncthreads();
  int pos = s_tmp[tid];
  for (int o = o0; o < min(o0 + per, 2 * N); ++o) {
    const int s = o / N, i = o - s * N;
    if ((ob[i] >> s) & 1) list_out[pos++] = o;
  }
  __syncthreads();
  return s_tmp[nt];
}

// Slot maps (ascending orbital order), particle-number and projection checks.
// commits: at load (stagger > 0) sample b's counter starts at b mod stagger so that about
// B / refresh_every samples re-factorise per commit call instead of the whole batch at
// once; after a refresh it restarts at 0.
__global__ void k_slots(Lattice lat, const int8_t* __restrict__ occ, const int32_t* __restrict__ list,
                        int32_t* __restrict__ orb_of_slot, int32_t* __restrict__ slot_of_orb,
                        int32_t* __restrict__ status, int32_t* __restrict__ commits, int stagger) {
  extern __shared__ int sm[];
  const int b = list ? list[blockIdx.x] : blockIdx.x;
  if (b < 0) return;
  const int N = lat.N, Ne = lat.Ne;
  int* olist = sm;               // [2N]
  int* tmp = sm + 2 * N;         // [blockDim + 1]
  __shared__ int s_up, s_dn, s_dbl;
  if (threadIdx.x == 0) { s_up = 0; s_dn = 0; s_dbl = 0; }
  __syncthreads();
  const int8_t* ob = occ + (size_t)b * N;
  int up = 0, dn = 0, dbl = 0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    up += ob[i] & 1;
    dn += (ob[i] >> 1) & 1;
    dbl += ob[i] == 3;
    if (ob[i] < 0 || ob[i] > 3) up += 1 << 20;  // invalid local state
  }
  atomicAdd(&s_up, up);
  atomicAdd(&s_dn, dn);
  atomicAdd(&s_dbl, dbl);
  const int n = occupied_list(ob, N, olist, tmp);
  int st = 0;
  if (s_up != lat.n_up || s_dn != lat.n_dn) st |= SCALE_SAMPLE_BAD_COUNT;
  if (lat.model == SCALE_MODEL_TJ && s_dbl > 0) st |= SCALE_SAMPLE_DOUBLE_OCC;
  for (int o = threadIdx.x; o < 2 * N; o += blockDim.x) slot_of_orb[(size_t)b * 2 * N + o] = -1;
  __syncthreads();
  if (st == 0) {
    for (int a = threadIdx.x; a < n && a < Ne; a += blockDim.x) {
      orb_of_slot[(size_t)b * Ne + a] = olist[a];
      slot_of_orb[(size_t)b * 2 * N + olist[a]] = a;
    }
  } else {
    for (int a = threadIdx.x; a < Ne; a += blockDim.x) orb_of_slot[(size_t)b * Ne + a] = -1;
  }
  if (threadIdx.x == 0) {
    status[b] = st;
    if (commits) commits[b] = stagger > 0 ? b % stagger : 0;
  }
}

// The orbital projection's parameters in precision TP.
template <typename TP>
struct Proj {
  int h;
  const TP* proj_w;  // [h][2Ne]
  const TP* proj_b;  // [2Ne]
  const TP* M0;      // [2N][Ne]
};

// Slater matrix in ascending orbital order (Sec. II.B "Orbital Projection"):
//   Phi[a][k] = M0[o_a][k] + proj_b[s*Ne+k] + sum_c H(L)_i[c] proj_w[c][s*Ne+k],
// o_a = s*N + i the a-th occupied orbital, from features H(L) of type TH, computed in TP and
// stored as FP64. The load and the refresh project in the mode's precision; the
// full-recompute path projects in FP64 (it divides two determinants, where an FP32 rounding
// of the entries would not cancel as the low-rank update's differences do).
template <typename TH, typename TP>
__global__ void k_phi(Lattice lat, Proj<TP> net, const int8_t* __restrict__ occ, const int32_t* __restrict__ list,
                      const TH* __restrict__ HL, double* __restrict__ phi, int B, const int32_t* __restrict__ count) {
  extern __shared__ int sm[];
  const int nrows = count ? min(*count, B) : B;
  for (int row = blockIdx.x; row < nrows; row += gridDim.x) {
  __syncthreads();  // the previous sample's use of shared memory is over
  const int b = list ? list[row] : row;
  if (b < 0) continue;
  const int N = lat.N, Ne = lat.Ne, h = net.h;
  int* olist = sm;
  int* tmp = sm + 2 * N;
  const int n = occupied_list(occ + (size_t)b * N, N, olist, tmp);
  double* P = phi + (size_t)b * Ne * Ne;
  if (n != Ne) {  // invalid sample: leave a zero matrix (singular)
    for (int q = threadIdx.x; q < Ne * Ne; q += blockDim.x) P[q] = 0.0;
    continue;
  }
  const TH* Hb = HL + (size_t)b * N * h;
  for (int q = threadIdx.x; q < Ne * Ne; q += blockDim.x) {
    const int a = q / Ne, k = q - a * Ne;
    const int o = olist[a], s = o / N, i = o - s * N;
    TP v = net.M0[(size_t)o * Ne + k] + net.proj_b[s * Ne + k];
    const TP* w = net.proj_w + s * Ne + k;
    const TH* x = Hb + (size_t)i * h;
    for (int c = 0; c < h; ++c) v += (TP)x[c] * w[(size_t)c * 2 * Ne];
    P[q] = (double)v;
  }
  }
}

// KE[t][n][d][c] = sum_c' E_t[n][c'] K_0[d][c'][c]: layer-0 response to the embedding of
// state n on site t, for every stencil offset d.
template <typename T>
__global__ void k_build_ke(Net<T> net, int Ns, T* __restrict__ KE) {
  const int h = net.h, kk = net.taps0;
  const size_t total = (size_t)Ns * 4 * kk * h;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int c = q % h;
    const int d = (q / h) % kk;
    const size_t tn = q / ((size_t)h * kk);  // t*4 + n
    const T* e = net.embed + tn * h;
    const T* w = net.kernel[0] + (size_t)d * h * h + c;
    T acc = T(0);
    for (int ci = 0; ci < h; ++ci) acc += e[ci] * w[(size_t)ci * h];
    KE[q] = acc;
  }
}

// log|psi| and sign in the ascending convention: sign = sign_slot * parity of the slot
// permutation orb_of_slot (inversions counted directly).
__global__ void k_logpsi_out(int Ne, const int32_t* __restrict__ orb_of_slot, const double* __restrict__ la_slot,
                             const int32_t* __restrict__ sg_slot, const int32_t* __restrict__ status,
                             double* __restrict__ logabs, int32_t* __restrict__ sign,
                             const int32_t* __restrict__ list) {
  const int b = list ? list[blockIdx.x] : blockIdx.x;
  const int32_t* os = orb_of_slot + (size_t)b * Ne;
  int inv = 0;
  for (int q = threadIdx.x; q < Ne * Ne; q += blockDim.x) {
    const int a = q / Ne, c = q - a * Ne;
    inv += (a < c) && (os[a] > os[c]);
  }
  __shared__ int s_inv;
  if (threadIdx.x == 0) s_inv = 0;
  __syncthreads();
  atomicAdd(&s_inv, inv);
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool bad = status[b] & (SCALE_SAMPLE_BAD_COUNT | SCALE_SAMPLE_DOUBLE_OCC | SCALE_SAMPLE_SINGULAR);
    const int sg = bad ? 0 : sg_slot[b] * ((s_inv & 1) ? -1 : 1);
    if (logabs) logabs[b] = bad ? -INFINITY : la_slot[b];
    if (sign) sign[b] = sg;
  }
}

// Site-wise layers 1..L-1 of every (sample, site) row on the tensor cores (mixed mode):
// one warp per 16 consecutive rows, activations kept in registers through the layers.
// Rows of samples not in the list are skipped.
template <int H, int KIND>
__global__ void __launch_bounds__(256) k_mlp_fwd(Net<float> net, const WFrag* __restrict__ wf, int N, int B,
                                                 const int32_t* __restrict__ list, const float* __restrict__ in,
                                                 float* __restrict__ out, const int32_t* __restrict__ count,
                                                 const float* __restrict__ oscale) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long row0 = (long long)warp * 16;
  // entries of the launch: B, or the first *count entries of a compacted list
  const long long rows = (long long)(count ? min(*count, B) : B) * N;
  if (row0 >= rows) return;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float x[H / 8][4];
  bool keep[2];
  long long drow[2];  // data row: sample (list entry or launch index) * N + site
#pragma unroll
  for (int hh = 0; hh < 2; ++hh) {
    const long long row = row0 + g + 8 * hh;
    bool k = row < rows;
    long long d = 0;
    if (k) {
      const long long q = row / N;
      const long long b = list ? (long long)list[q] : q;
      k = b >= 0;
      d = b * N + (row - q * N);
    }
    keep[hh] = k;
    drow[hh] = d;
  }
#pragma unroll
  for (int j = 0; j < H / 8; ++j) {
    const int c = 8 * j + 2 * t;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      x[j][2 * hh] = keep[hh] ? in[drow[hh] * H + c] : 0.f;
      x[j][2 * hh + 1] = keep[hh] ? in[drow[hh] * H + c + 1] : 0.f;
    }
  }
  mlp_tile<H, KIND>(x, wf, net.bias, net.resid, net.L, net.act, oscale);
#pragma unroll
  for (int j = 0; j < H / 8; ++j) {
    const int c = 8 * j + 2 * t;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      if (keep[hh]) {
        out[drow[hh] * H + c] = x[j][2 * hh];
        out[drow[hh] * H + c + 1] = x[j][2 * hh + 1];
      }
    }
  }
}

// kFP16 scaling of the site-wise layers (l >= 1): with max|W_l| = f 2^e_l, f in [1/2, 1), the
// fragments hold W_l 2^-e_l and the layer's accumulator is multiplied back by 2^e_l / 2^4
// (both exact). One block per layer.
__global__ void k_fp16_scales(Net<float> net, float* __restrict__ sc) {
  const int l = blockIdx.x;
  __shared__ float red[32];
  float m = 0.f;
  if (l >= 1 && net.ksize[l] == 1) {
    const float* W = net.kernel[l];
    for (int q = threadIdx.x; q < net.h * net.h; q += blockDim.x) m = fmaxf(m, fabsf(W[q]));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    int e = 0;
    if (m > 0.f && isfinite(m)) frexpf(m, &e);
    sc[l] = ldexpf(1.f, -e);
    sc[kMaxLayers + l] = ldexpf(1.f, e) / kFp16InScale;
  }
}

// hi/lo fragments of the site-wise weights W_l[c_in][c_out] (layers l >= 1):
//   BF16 / FP16: b0 = (W[16kk + 2t][8j + g], W[16kk + 2t + 1][8j + g]), b1 = the same at rows + 8
//                (FP16: W scaled by wsc[l]);
//   TF32: b0 = W[8kk + 2t][8j + g], b1 = W[8kk + 2t + 1][8j + g] (permuted k, see mlp_mma.cuh).
template <int H, int KIND>
__global__ void k_build_wfrag(Net<float> net, WFrag* __restrict__ wf, const float* __restrict__ wsc) {
  constexpr int NT = MmaShape<H, KIND>::NT, KT = MmaShape<H, KIND>::KT;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int total = net.L * KT * NT * 32;
  if (q >= total) return;
  const int lane = q & 31, j = (q >> 5) % NT, kk = (q >> 5) / NT % KT, l = (q >> 5) / (NT * KT);
  WFrag f{};
  if (l >= 1 && net.ksize[l] == 1) {
    const int g = lane >> 2, t = lane & 3;
    const float* W = net.kernel[l];
    const int n = 8 * j + g;
    if constexpr (KIND == kTF32) {
      const int k0 = 8 * kk + 2 * t;
      split_tf32(W[(size_t)k0 * H + n], f.v[0], f.v[2]);
      split_tf32(W[(size_t)(k0 + 1) * H + n], f.v[1], f.v[3]);
    } else if constexpr (KIND == kFP16) {
      const int k0 = 16 * kk + 2 * t;
      const float sw = wsc[l];
      split2h(sw * W[(size_t)k0 * H + n], sw * W[(size_t)(k0 + 1) * H + n], f.v[0], f.v[2]);
      split2h(sw * W[(size_t)(k0 + 8) * H + n], sw * W[(size_t)(k0 + 9) * H + n], f.v[1], f.v[3]);
    } else {
      const int k0 = 16 * kk + 2 * t;
      split2(W[(size_t)k0 * H + n], W[(size_t)(k0 + 1) * H + n], f.v[0], f.v[2]);
      split2(W[(size_t)(k0 + 8) * H + n], W[(size_t)(k0 + 9) * H + n], f.v[1], f.v[3]);
    }
  }
  wf[q] = f;
}

// Arguments of k_mlp_fwd, and its launch at the context's channel capacity.
struct MlpFwdArgs {
  Net<float> net;
  const WFrag* wf;
  int N, B;
  const int32_t* list;
  const float* in;
  float* out;
  const int32_t* count;
  const float* oscale;
};
template <int KIND>
void launch_mlp_fwd(const scale_ctx* c, int blocks, const MlpFwdArgs& f) {
  if (c->hpad == 16)
    k_mlp_fwd<16, KIND><<<blocks, 256, 0, c->stream>>>(f.net, f.wf, f.N, f.B, f.list, f.in, f.out, f.count, f.oscale);
  else if (c->hpad == 32)
    k_mlp_fwd<32, KIND><<<blocks, 256, 0, c->stream>>>(f.net, f.wf, f.N, f.B, f.list, f.in, f.out, f.count, f.oscale);
  else
    k_mlp_fwd<64, KIND><<<blocks, 256, 0, c->stream>>>(f.net, f.wf, f.N, f.B, f.list, f.in, f.out, f.count, f.oscale);
}

// occ rows of a packed batch into the listed samples' rows.
__global__ void k_scatter_occ(int N, const int8_t* __restrict__ src, const int32_t* __restrict__ list,
                              int8_t* __restrict__ dst) {
  const int w = blockIdx.x, b = list[w];
  for (int i = threadIdx.x; i < N; i += blockDim.x) dst[(size_t)b * N + i] = src[(size_t)w * N + i];
}

}  // namespace

template <int KIND>
void build_wfrag_k(scale_ctx* c) {
  const Net<float> net = make_net<float>(c);
  const int total = c->L * (KIND == kTF32 ? c->hpad / 8 : c->hpad / 16) * (c->hpad / 8) * 32;
  const int blocks = (total + 255) / 256;
  const float* wsc = nullptr;
  if constexpr (KIND == kFP16) {
    float* sc = fp16_scales(c);
    k_fp16_scales<<<c->L, 256, 0, c->stream>>>(net, sc);
    wsc = sc;
  }
  if (c->hpad == 16) k_build_wfrag<16, KIND><<<blocks, 256, 0, c->stream>>>(net, (WFrag*)c->wfrag, wsc);
  else if (c->hpad == 32) k_build_wfrag<32, KIND><<<blocks, 256, 0, c->stream>>>(net, (WFrag*)c->wfrag, wsc);
  else k_build_wfrag<64, KIND><<<blocks, 256, 0, c->stream>>>(net, (WFrag*)c->wfrag, wsc);
}

cudaError_t launch_build_wfrag(scale_ctx* c) {
  if (!c->use_mma) return cudaSuccess;
  const int kind = mma_kind_of(c->arch.precision);
  if (kind == kBF16) build_wfrag_k<kBF16>(c);
  else if (kind == kFP16) build_wfrag_k<kFP16>(c);
  else build_wfrag_k<kTF32>(c);
  return cudaGetLastError();
}

template <typename T>
Net<T> make_net(scale_ctx* c) {
  Net<T> n{};
  n.h = c->h;
  n.L = c->L;
  n.act = c->arch.act;
  n.per_site = c->arch.per_site_embed;
  n.stencil = c->arch.stencil;
  n.taps0 = stencil_taps(c->arch.stencil, c->arch.ksize[0]);
  const T* base = c->fp64 ? (const T*)c->params64 : (const T*)c->params32;
  int64_t p = 0;
  n.embed = base + p;
  p += (int64_t)(c->arch.per_site_embed ? c->N : 1) * 4 * c->h;
  for (int l = 0; l < c->L; ++l) {
    n.ksize[l] = c->arch.ksize[l];
    n.resid[l] = c->arch.residual[l];
    n.kernel[l] = base + p;  // [taps][h][h]: the stencil's taps in row-major box order
    p += (int64_t)stencil_taps(c->arch.stencil, n.ksize[l]) * c->h * c->h;
    n.bias[l] = base + p;
    p += c->h;
  }
  n.proj_w = base + p;
  p += (int64_t)c->h * 2 * c->Ne;
  n.proj_b = base + p;
  n.M0 = c->fp64 ? (const T*)c->M0_64 : (const T*)c->M0_32;
  n.M0b = (const T*)c->M0b;
  n.KE = (const T*)c->KE;
  return n;
}

template Net<double> make_net<double>(scale_ctx*);
template Net<float> make_net<float>(scale_ctx*);

namespace {
template <typename T>
cudaError_t forward_t(scale_ctx* c, const int8_t* occ, int B, const int32_t* list, bool keep_cache,
                      double* phi_out, const int32_t* count, bool proj64) {
  const Net<T> net = make_net<T>(c);
  const int N = c->N, h = c->h;
  // with a compacted list (count on the device) the kernels loop over its entries from a
  // capped grid instead of launching a CTA per sample of the batch
  const int Bgrid = count ? std::min(B, 256) : B;
  dim3 grid((N * h + 127) / 128, Bgrid);
  T* bufs[2] = {(T*)c->act_a, (T*)c->act_b};
  const T* in = nullptr;
  const bool mma = c->use_mma && c->L > 1;
  for (int l = 0; l < (mma ? 1 : c->L); ++l) {
    T* out = (l == c->L - 1 && keep_cache) ? (T*)c->HL : bufs[l & 1];
    T* zo = (l == 0 && keep_cache) ? (T*)c->z0 : nullptr;
    k_layer<T><<<grid, 128, 0, c->stream>>>(c->lat, net, l, occ, list, in, out, zo, B, count);
    in = out;
  }
  if constexpr (sizeof(T) == 4) {
    if (mma) {
      float* out = keep_cache ? (float*)c->HL : (float*)bufs[1];
      const long long tiles = ((long long)B * N + 15) / 16;
      const int blocks = (int)((tiles + 7) / 8);
      const Net<float> nf = make_net<float>(c);
      const WFrag* wf = (const WFrag*)c->wfrag;
      const float* fin = (const float*)in;
      const int kind = mma_kind_of(c->arch.precision);
      const float* osc = kind == kFP16 ? fp16_scales(c) + kMaxLayers : nullptr;
      const MlpFwdArgs fa{nf, wf, N, B, list, fin, out, count, osc};
      if (kind == kBF16) launch_mlp_fwd<kBF16>(c, blocks, fa);
      else if (kind == kFP16) launch_mlp_fwd<kFP16>(c, blocks, fa);
      else launch_mlp_fwd<kTF32>(c, blocks, fa);
      in = (const T*)out;
    }
  }
  const size_t smem = sizeof(int) * (2 * N + 257);
  const int Bphi = count ? std::min(B, 1024) : B;
  if (phi_out) {
    if (proj64 && !c->fp64) {
      // FP64 projection parameters: the flat FP64 vector at the offsets of make_net
      const int64_t off_w = (const T*)net.proj_w - (const T*)c->params32;
      const Proj<double> p64{c->h, c->params64 + off_w, c->params64 + off_w + (int64_t)c->h * 2 * c->Ne, c->M0_64};
      k_phi<T, double><<<Bphi, 256, smem, c->stream>>>(c->lat, p64, occ, list, in, phi_out, B, count);
    } else {
      const Proj<T> pt{c->h, net.proj_w, net.proj_b, net.M0};
      k_phi<T, T><<<Bphi, 256, smem, c->stream>>>(c->lat, pt, occ, list, in, phi_out, B, count);
    }
  }
  return cudaGetLastError();
}
}  // namespace

// Forward every listed sample of occ; keep_cache writes z0 / HL of the context.
cudaError_t launch_forward(scale_ctx* c, const int8_t* occ, int B, const int32_t* list, bool keep_cache,
                           double* phi_out, const int32_t* count) {
  if (c->ace) {  // ACE / wide: whole batches only (no list); the wide cache keeps H(L)
    if (list || count || !phi_out) return cudaErrorInvalidValue;
    return launch_ace_forward(c, occ, B, phi_out, nullptr, keep_cache && c->wide_lr ? c->HL : nullptr);
  }
  if (c->fp64) return forward_t<double>(c, occ, B, list, keep_cache, phi_out, count, false);
  return forward_t<float>(c, occ, B, list, keep_cache, phi_out, count, false);
}

// Forward for the full-recompute path: FP64 Slater matrices of B packed configurations into
// phi [B][Ne][Ne] (the network in the mode's precision); features go to the scratch buffers.
// Entries with list[g] < 0 are skipped (SCALE family); the ACE and wide networks evaluate
// the first *vcount configurations (the valid entries of a chunk form a prefix).
cudaError_t launch_forward_phi(scale_ctx* c, const int8_t* occ, int B, const int32_t* list, const int32_t* vcount,
                               double* phi) {
  if (c->ace) return launch_ace_forward(c, occ, B, phi, vcount);
  if (c->fp64) return forward_t<double>(c, occ, B, list, false, phi, nullptr, true);
  return forward_t<float>(c, occ, B, list, false, phi, nullptr, true);
}

cudaError_t launch_slots(scale_ctx* c, const int8_t* occ, int B) {
  const size_t smem = sizeof(int) * (2 * c->N + 257);
  k_slots<<<B, 256, smem, c->stream>>>(c->lat, occ, nullptr, c->orb_of_slot, c->slot_of_orb, c->status,
                                        c->commits, c->arch.refresh_every);
  return cudaGetLastError();
}

cudaError_t launch_slots_list(scale_ctx* c, const int32_t* list, int B) {
  const size_t smem = sizeof(int) * (2 * c->N + 257);
  k_slots<<<B, 256, smem, c->stream>>>(c->lat, c->occ, list, c->orb_of_slot, c->slot_of_orb, c->status,
                                        c->commits, 0);
  return cudaGetLastError();
}

cudaError_t launch_build_ke(scale_ctx* c) {
  const int Ns = c->arch.per_site_embed ? c->N : 1;
  const size_t total = (size_t)Ns * 4 * stencil_taps(c->arch.stencil, c->k0) * c->h;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 4096);
  if (c->fp64)
    k_build_ke<double><<<blocks, 256, 0, c->stream>>>(make_net<double>(c), Ns, (double*)c->KE);
  else
    k_build_ke<float><<<blocks, 256, 0, c->stream>>>(make_net<float>(c), Ns, (float*)c->KE);
  return cudaGetLastError();
}

cudaError_t launch_logpsi_out(scale_ctx* c, double* logabs, int32_t* sign) {
  k_logpsi_out<<<c->B, 256, 0, c->stream>>>(c->Ne, c->orb_of_slot, c->logabs, c->sign_slot, c->status,
                                             logabs, sign, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_logpsi_list(scale_ctx* c, const int32_t* list, int n, double* logabs, int32_t* sign) {
  k_logpsi_out<<<n, 256, 0, c->stream>>>(c->Ne, c->orb_of_slot, c->logabs, c->sign_slot, c->status, logabs, sign,
                                         list);
  return cudaGetLastError();
}

// Load the packed configurations occ[n][N] into the listed samples and build their cache
// (slot maps, forward, FP64 inverse, projector) -- the load sequence restricted to a list.
cudaError_t launch_load_list(scale_ctx* c, const int8_t* occ, const int32_t* list, int n) {
  cudaError_t e;
  k_scatter_occ<<<n, 128, 0, c->stream>>>(c->N, occ, list, c->occ);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_slots_list(c, list, n)) != cudaSuccess) return e;
  if ((e = launch_forward(c, c->occ, n, list, true, c->Phi64)) != cudaSuccess) return e;
  if ((e = launch_gj(c, c->Phi64, c->Ne, n, list, true, c->fp64, c->Binv, c->logabs, c->sign_slot, c->status)) !=
      cudaSuccess)
    return e;
  return launch_projector(c, n, list);
}

}  // namespace scale
