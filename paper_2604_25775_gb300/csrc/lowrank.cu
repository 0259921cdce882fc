// lowrank.cu -- local energies and amplitude ratios by the cached-network + rank-r
// determinant update of Sec. II.C, and the projector P_s = W_s Phi^-1 it relies on.
//
// One CTA per sample. Connected configurations are enumerated on the device in the fixed
// order of eloc_common.cuh, compacted chunk by chunk, and handed to the warps (one move per
// warp at a time, move.cuh). Per-move contributions are summed in enumeration order, so E_loc
// does not depend on scheduling. (Mixed precision at the tensor-core widths runs the batched
// kernel of eloc_tc.cu instead.)
//
// Matrix elements in slot order (a moved electron keeps its determinant row):
//   hop     -t (NN) / -t' (NNN) times det R   (its Jordan-Wigner sign and the row
//           permutation sign of the ascending convention cancel),
//   exchange (J/2)(S+_i S-_j + h.c.) = -(J/2) (c+_{i up} c_{j up})(c+_{j dn} c_{i dn}):
//           -J/2 times det R.
// Diagonal: Hubbard U * (doubly occupied sites); t-J J sum_<ij> Sz_i Sz_j; the
// particle-hole transformed Hubbard model U sum_i n_up (1 - n_dn).
#include <algorithm>

#include "eloc_common.cuh"

namespace scale {

namespace {

constexpr int kWarps = 8;

// WARPS warps per sample; the sample's cached rows (Binv, Pt, z0, H(L)) are read through
// L1/L2, shared memory holds the per-warp move scratch and the move list.
template <typename T, int H, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_eloc(LowrankArgs a, Net<T> net) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = a.lat.N, Ne = a.lat.Ne, h = net.h;
  MoveScratch<T, H>* ms_all = reinterpret_cast<MoveScratch<T, H>*>(smem);
  uint32_t* mlist = reinterpret_cast<uint32_t*>(ms_all + WARPS);     // [kMoveChunk]
  double* contrib = reinterpret_cast<double*>(mlist + kMoveChunk);   // [kMoveChunk]
  int32_t* slot_s = reinterpret_cast<int32_t*>(contrib + kMoveChunk);
  int8_t* occ_s = reinterpret_cast<int8_t*>(slot_s + 2 * N);
  __shared__ int warp_cnt[WARPS];
  __shared__ double s_diag;
  __shared__ int s_next;

  const int b = a.list ? a.list[blockIdx.x] : blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int st = a.status[b];
  if (st & (SCALE_SAMPLE_BAD_COUNT | SCALE_SAMPLE_DOUBLE_OCC | SCALE_SAMPLE_SINGULAR)) {
    if (tid == 0) {
      a.out[b] = CUDART_NAN;
      if (a.move_count) a.move_count[b] = 0;
    }
    return;
  }
  for (int i = tid; i < N; i += blockDim.x) occ_s[i] = a.occ[(size_t)b * N + i];
  for (int o = tid; o < 2 * N; o += blockDim.x) slot_s[o] = a.slot_of_orb[(size_t)b * 2 * N + o];
  __syncthreads();
  if (tid == 0) s_diag = diag_energy(a, occ_s);
  SampleView<T> sv;
  sv.occ = occ_s;
  sv.slot_of_orb = slot_s;
  sv.z0 = (const T*)a.z0 + (size_t)b * N * h;
  sv.HL = (const T*)a.HL + (size_t)b * N * h;
  sv.Binv = (const T*)a.Binv + (size_t)b * Ne * Ne;
  sv.Pt = (const T*)a.Pt + (size_t)b * 2 * Ne * h;
  sv.G0t = (const T*)a.G0t + (size_t)b * Ne * 2 * N;
  MoveScratch<T, H>& ms = ms_all[warp];

  const int ncand = candidate_count(a);
  double total = 0.0;  // thread 0
  int nmoves = 0;
  for (int cs = 0; cs < ncand; cs += kMoveChunk) {
    const int ce = min(ncand, cs + kMoveChunk);
    // enumerate and compact the allowed moves of this chunk (enumeration order)
    const int nm = enumerate_chunk<WARPS>(a, occ_s, cs, ce, mlist, warp_cnt);
    if (tid == 0) s_next = 0;
    __syncthreads();
    // warps take the next move as they finish the previous one
    for (;;) {
      int mi = 0;
      if (lane == 0) mi = atomicAdd(&s_next, 1);
      mi = __shfl_sync(0xffffffffu, mi, 0);
      if (mi >= nm) break;
      const uint32_t pm = mlist[mi];
      if (lane == 0) {
        const MoveDesc m = unpack_move(pm);
        ms.src = m.src;
        ms.dst = m.dst;
        ms.spin = m.spin;
        ms.kind = m.kind;
      }
      __syncwarp();
      move_features<T, H>(a.lat, net, a.k0, sv, a.mf, ms);
      const int r = move_matrix<T, H>(a.lat, net, sv, ms);
      const T det = (r < 0) ? T(CUDART_NAN) : warp_det<T, H>(ms, r);
      if (lane == 0) contrib[mi] = move_coeff(a.lat, pm) * (double)det;
      __syncwarp();
    }
    __syncthreads();
    // fixed-order sum of the chunk: lane l adds contributions l, l+32, ..., then an xor tree
    // (both orders independent of which warp evaluated which move)
    if (warp == 0) {
      double s = 0.0;
      for (int q = lane; q < nm; q += 32) s += contrib[q];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (lane == 0) {
        total += s;
        nmoves += nm;
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    a.out[b] = s_diag + total;
    if (a.move_count) a.move_count[b] = nmoves;
  }
}

// psi(n')/psi(n) in the ascending convention for M explicit moves per sample.
template <typename T, int H>
__global__ void __launch_bounds__(kWarps * 32) k_ratios(LowrankArgs a, Net<T> net) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = a.lat.N, Ne = a.lat.Ne, h = net.h;
  MoveScratch<T, H>* ms_all = reinterpret_cast<MoveScratch<T, H>*>(smem);
  int32_t* slot_s = reinterpret_cast<int32_t*>(ms_all + kWarps);
  int8_t* occ_s = reinterpret_cast<int8_t*>(slot_s + 2 * N);
  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int st = a.status[b];
  const bool bad = st & (SCALE_SAMPLE_BAD_COUNT | SCALE_SAMPLE_DOUBLE_OCC | SCALE_SAMPLE_SINGULAR);
  if (bad) {
    for (int m = tid; m < a.M; m += blockDim.x) a.out[(size_t)b * a.M + m] = CUDART_NAN;
    return;
  }
  for (int i = tid; i < N; i += blockDim.x) occ_s[i] = a.occ[(size_t)b * N + i];
  for (int o = tid; o < 2 * N; o += blockDim.x) slot_s[o] = a.slot_of_orb[(size_t)b * 2 * N + o];
  __syncthreads();
  SampleView<T> sv;
  sv.occ = occ_s;
  sv.slot_of_orb = slot_s;
  sv.z0 = (const T*)a.z0 + (size_t)b * N * h;
  sv.HL = (const T*)a.HL + (size_t)b * N * h;
  sv.Binv = (const T*)a.Binv + (size_t)b * Ne * Ne;
  sv.Pt = (const T*)a.Pt + (size_t)b * 2 * Ne * h;
  sv.G0t = (const T*)a.G0t + (size_t)b * Ne * 2 * N;
  MoveScratch<T, H>& ms = ms_all[warp];
  for (int mi = warp; mi < a.M; mi += kWarps) {
    const int32_t* mv = a.moves + ((size_t)b * a.M + mi) * 4;
    const int kind = mv[0], src = mv[1], dst = mv[2], spin = mv[3];
    double out;
    if (kind < 0) {
      out = 1.0;
    } else if (!move_allowed(a.lat, kind, src, dst, spin, occ_s)) {
      out = 0.0;
    } else {
      if (lane == 0) {
        ms.kind = kind;
        ms.src = src;
        ms.dst = dst;
        ms.spin = spin;
      }
      __syncwarp();
      move_features<T, H>(a.lat, net, a.k0, sv, a.mf, ms);
      const int r = move_matrix<T, H>(a.lat, net, sv, ms);
      const T det = (r < 0) ? T(CUDART_NAN) : warp_det<T, H>(ms, r);
      int par;
      if (kind == 0) {
        par = between_parity(occ_s, N, spin * N + src, spin * N + dst);
      } else {
        // exchange: the up electron and the down electron each hop between src and dst
        par = between_parity(occ_s, N, src, dst) ^ between_parity(occ_s, N, N + src, N + dst);
      }
      out = (par ? -1.0 : 1.0) * (double)det;
    }
    if (lane == 0) a.out[(size_t)b * a.M + mi] = out;
    __syncwarp();
  }
}

// Pt[s][c][:] = W_s Binv[c], i.e. the GEMM Pt[s] = Binv (Ne x Ne) * W_s^T (Ne x h),
// W_s^T[k][cc] = proj_w[cc][s*Ne + k]. 32 rows per CTA, K tiles of 32.
template <typename T>
__global__ void __launch_bounds__(256) k_project(int Ne, int h, const T* __restrict__ proj_w,
                                                 const T* __restrict__ Binv, T* __restrict__ Pt,
                                                 const int32_t* __restrict__ list, int B,
                                                 const int32_t* __restrict__ count) {
  __shared__ T Bs[32][33];
  __shared__ T Ws[32][2 * kMaxH + 1];
  const int nrows = count ? min(*count, B) : B;  // a compacted list: its first *count entries
  for (int lrow = blockIdx.y; lrow < nrows; lrow += gridDim.y) {
  __syncthreads();  // the previous sample's tiles are consumed
  const int b = list ? list[lrow] : lrow;
  if (b < 0) continue;
  const int c0 = blockIdx.x * 32;
  const int tid = threadIdx.x;
  const int row = tid >> 3, grp = tid & 7;
  const int ncol = 2 * h;
  T acc[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) acc[u] = T(0);
  const T* Bb = Binv + (size_t)b * Ne * Ne;
  for (int k0 = 0; k0 < Ne; k0 += 32) {
    for (int q = tid; q < 32 * 32; q += 256) {
      const int rr = q >> 5, kk = q & 31;
      const int c = c0 + rr, k = k0 + kk;
      Bs[rr][kk] = (c < Ne && k < Ne) ? Bb[(size_t)c * Ne + k] : T(0);
    }
    for (int q = tid; q < 32 * ncol; q += 256) {
      const int kk = q / ncol, col = q - kk * ncol;
      const int s = col / h, cc = col - s * h, k = k0 + kk;
      Ws[kk][col] = (k < Ne) ? proj_w[(size_t)cc * 2 * Ne + s * Ne + k] : T(0);
    }
    __syncthreads();
    for (int kk = 0; kk < 32; ++kk) {
      const T bv = Bs[row][kk];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int col = grp + 8 * u;
        if (col < ncol) acc[u] += bv * Ws[kk][col];
      }
    }
    __syncthreads();
  }
  const int c = c0 + row;
  if (c < Ne) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int col = grp + 8 * u;
      if (col < ncol) {
        const int s = col / h, cc = col - s * h;
        Pt[(((size_t)b * 2 + s) * Ne + c) * h + cc] = acc[u];
      }
    }
  }
  }
}

template <typename T, int H, int WARPS>
size_t eloc_smem(int N) {
  return sizeof(MoveScratch<T, H>) * WARPS + (sizeof(uint32_t) + sizeof(double)) * kMoveChunk +
         sizeof(int32_t) * 2 * N + N + 16;
}

template <typename T, int H>
size_t ratio_smem(int N) {
  return sizeof(MoveScratch<T, H>) * kWarps + sizeof(int32_t) * 2 * N + N + 16;
}


template <typename T, int H, int WARPS>
cudaError_t eloc_launch(scale_ctx* c, const LowrankArgs& a, int n) {
  const size_t smem = eloc_smem<T, H, WARPS>(c->N);
  cudaError_t e = cudaFuncSetAttribute(k_eloc<T, H, WARPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_eloc<T, H, WARPS><<<n, WARPS * 32, smem, c->stream>>>(a, make_net<T>(c));
  return cudaGetLastError();
}

// Launch shape: the most warps per CTA (one CTA per SM) whose move scratch fits, up to 20.
// Measured at 16x16, 8192 walkers: 20 warps 65.7 ms, 22 warps 68.8 ms (too little L1 left
// for the cached rows), 16 warps 77.7 ms, 12 warps 88.0 ms; staging the projector in shared
// memory instead (16 warps) took 80.1 ms.
template <typename T, int H>
cudaError_t eloc_t(scale_ctx* c, double* eloc, const int32_t* list, int n) {
  LowrankArgs a = make_args(c);
  a.out = eloc;
  a.move_count = c->move_count;
  a.list = list;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (eloc_smem<T, H, 20>(c->N) <= (size_t)optin) return eloc_launch<T, H, 20>(c, a, n);
  if (eloc_smem<T, H, 16>(c->N) <= (size_t)optin) return eloc_launch<T, H, 16>(c, a, n);
  if (eloc_smem<T, H, 12>(c->N) <= (size_t)optin) return eloc_launch<T, H, 12>(c, a, n);
  if (eloc_smem<T, H, 8>(c->N) <= (size_t)optin) return eloc_launch<T, H, 8>(c, a, n);
  return eloc_launch<T, H, 4>(c, a, n);  // FP64 with 64 channels: 28 KB of move scratch per warp
}

template <typename T, int H>
cudaError_t ratios_t(scale_ctx* c, const int32_t* moves, int M, double* ratio) {
  LowrankArgs a = make_args(c);
  a.out = ratio;
  a.moves = moves;
  a.M = M;
  const size_t smem = ratio_smem<T, H>(c->N);
  cudaError_t e = cudaFuncSetAttribute(k_ratios<T, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_ratios<T, H><<<c->B, kWarps * 32, smem, c->stream>>>(a, make_net<T>(c));
  return cudaGetLastError();
}

// G0t[b][j][o] = (M0[o] + proj_b[s(o)]) . Binv[b][j]: the part of every Slater row's
// product with the inverse that does not depend on the network features (the moved rows of
// R need it for the target orbital). A GEMM per sample: CTA tiles of 64 slots x 64 orbitals,
// 4 x 4 per thread, K staged 32 at a time through shared memory; the listed samples only
// (their first *count entries when count is given).
template <typename T>
__global__ void __launch_bounds__(256) k_build_g0(int Ne, int No, const T* __restrict__ Binv,
                                                  const T* __restrict__ M0b, T* __restrict__ G0t,
                                                  const int32_t* __restrict__ list, int B,
                                                  const int32_t* __restrict__ count) {
  __shared__ T As[32][65];  // As[k][j] = Binv[j][k]
  __shared__ T Ms[32][65];  // Ms[k][o] = M0b[o][k]
  const int nrows = count ? min(*count, B) : B;
  const int j0 = blockIdx.x * 64, o0 = blockIdx.y * 64;
  const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
  for (int lrow = blockIdx.z; lrow < nrows; lrow += gridDim.z) {
    const int b = list ? list[lrow] : lrow;
    if (b < 0) continue;
    const T* Bb = Binv + (size_t)b * Ne * Ne;
    T acc[4][4] = {};
    for (int k0 = 0; k0 < Ne; k0 += 32) {
      __syncthreads();  // the previous tiles are consumed
      for (int q = tid; q < 64 * 32; q += 256) {
        const int rr = q >> 5, kk = q & 31, k = k0 + kk;
        As[kk][rr] = (j0 + rr < Ne && k < Ne) ? Bb[(size_t)(j0 + rr) * Ne + k] : T(0);
        Ms[kk][rr] = (o0 + rr < No && k < Ne) ? M0b[(size_t)(o0 + rr) * Ne + k] : T(0);
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < 32; ++kk) {
        T x[4], y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          x[u] = As[kk][tr + 16 * u];
          y[u] = Ms[kk][tc + 16 * u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] += x[u] * y[v];
      }
    }
    T* out = G0t + (size_t)b * Ne * No;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = j0 + tr + 16 * u;
      if (j >= Ne) continue;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int o = o0 + tc + 16 * v;
        if (o < No) out[(size_t)j * No + o] = acc[u][v];
      }
    }
  }
}

template <typename T>
cudaError_t build_g0_t(scale_ctx* c, int B, const int32_t* list, const int32_t* count) {
  const int No = 2 * c->N;
  const dim3 g0grid((c->Ne + 63) / 64, (No + 63) / 64, count ? std::min(B, 256) : std::min(B, 65535));
  k_build_g0<T><<<g0grid, 256, 0, c->stream>>>(c->Ne, No, (const T*)c->Binv, (const T*)c->M0b, (T*)c->G0t, list, B,
                                               count);
  return cudaGetLastError();
}

template <typename T>
cudaError_t project_t(scale_ctx* c, int B, const int32_t* list, const int32_t* count) {
  dim3 grid((c->Ne + 31) / 32, count ? std::min(B, 1024) : B);
  k_project<T><<<grid, 256, 0, c->stream>>>(c->Ne, c->h, make_net<T>(c).proj_w, (const T*)c->Binv, (T*)c->Pt, list,
                                            B, count);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return build_g0_t<T>(c, B, list, count);
}

}  // namespace

#define SCALE_DISPATCH_H(c, FN, ...)                                                          \
  ((c)->hpad == 16   ? ((c)->fp64 ? FN<double, 16>(__VA_ARGS__) : FN<float, 16>(__VA_ARGS__)) \
   : (c)->hpad == 32 ? ((c)->fp64 ? FN<double, 32>(__VA_ARGS__) : FN<float, 32>(__VA_ARGS__)) \
                     : ((c)->fp64 ? FN<double, 64>(__VA_ARGS__) : FN<float, 64>(__VA_ARGS__)))

// Mixed precision at 32 channels runs the batched tensor-core kernel (eloc_tc.cu); every
// other shape the per-warp kernel above.
cudaError_t launch_eloc_lowrank(scale_ctx* c, double* eloc) {
  if (c->et_wimg) return launch_eloc_tc(c, eloc, nullptr, c->B);
  return SCALE_DISPATCH_H(c, eloc_t, c, eloc, nullptr, c->B);
}

// E_loc of the listed samples only (outputs indexed by sample).
cudaError_t launch_eloc_lowrank_list(scale_ctx* c, const int32_t* list, int n, double* eloc) {
  if (c->et_wimg) return launch_eloc_tc(c, eloc, list, n);
  return SCALE_DISPATCH_H(c, eloc_t, c, eloc, list, n);
}

cudaError_t launch_ratios(scale_ctx* c, const int32_t* moves, int M, double* ratio) {
  return SCALE_DISPATCH_H(c, ratios_t, c, moves, M, ratio);
}

cudaError_t launch_projector(scale_ctx* c, int B, const int32_t* list, const int32_t* count) {
  return c->fp64 ? project_t<double>(c, B, list, count) : project_t<float>(c, B, list, count);
}

cudaError_t launch_build_g0(scale_ctx* c, int B, const int32_t* list, const int32_t* count) {
  return c->fp64 ? build_g0_t<double>(c, B, list, count) : build_g0_t<float>(c, B, list, count);
}

}  // namespace scale
