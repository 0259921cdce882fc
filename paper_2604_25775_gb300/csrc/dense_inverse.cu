// dense_inverse.cu -- batched Gauss-Jordan elimination with partial pivoting.
//
// One CTA per matrix. It returns log|det|, the sign and (inverse mode) the inverse in the
// library's dual-row layout Binv[c][k] = (A^-1)[k][c]; "det-only" mode restricts the
// elimination to the rows not yet pivoted and the columns to the right, which is LU with
// partial pivoting (n^3/3 multiply-adds) -- both are the "single LU decomposition" of
// Sec. II.C giving the determinant and the inverse together.
//
// Blocking. Pivots are taken W columns at a time. The W-column panel is swept in shared
// memory; the W elementary row operations of the block combine into T = I + U P^T, where
// the columns of U are the swept panel columns minus the unit vectors of the pivot rows
// and P selects the pivot rows. Every other column then takes one rank-W update
//     A[i][c] += sum_j U[i][j] A_old[p_j][c]
// so each matrix element is read and written once per W pivots. The matrix stays in
// global memory (L2-resident while the CTAs in flight fit), the work is the FMA pipe of
// the working type; on sm_103a FP64 this kernel is DFMA-bound.
//
// Pivot choice: largest |value| among unpivoted rows, ties to the lowest row index.
// Pivoting is implicit (no row swaps); the pivot row of column k is p[k] and the final
// storage holds A^-1[k][p[j]] at (p[k], j).
#include <cooperative_groups.h>

#include <algorithm>

#include "scale_internal.cuh"

namespace cg = cooperative_groups;

namespace scale {

namespace {

constexpr int kThreads = 1024;  // 32 warps: DFMA latency hidden within one CTA (refresh batches
                                 // are often one CTA per SM)

template <typename TW>
struct ArgMax {
  TW v;
  int i;
};

// Pivot search on integer keys: the bit pattern of |x| orders like |x| (and puts NaN above
// every number), so the search runs on the integer pipe instead of FP64 compares.
template <typename TW>
struct AbsKey;
template <>
struct AbsKey<double> {
  using T = unsigned long long;
  __device__ static T of(double x) { return (T)__double_as_longlong(x) & 0x7fffffffffffffffull; }
};
template <>
struct AbsKey<float> {
  using T = unsigned int;
  __device__ static T of(float x) { return (T)__float_as_uint(x) & 0x7fffffffu; }
};
template <typename K>
__device__ __forceinline__ void key_merge(K& k, int& i, K k2, int i2) {
  if (k2 > k || (k2 == k && i2 < i)) {
    k = k2;
    i = i2;
  }
}

// Largest key over the warp (ties to the lowest row); the result is valid on lane 0.
template <typename K>
__device__ __forceinline__ void warp_key_max(K& k, int& i) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const K k2 = __shfl_down_sync(0xffffffffu, k, off);
    const int i2 = __shfl_down_sync(0xffffffffu, i, off);
    key_merge(k, i, k2, i2);
  }
}

// Pivot row of panel column jj: the largest |value| among the rows not yet pivoted, ties to
// the lowest row. Each thread scans its rows, each warp merges its lanes, and warp 0 merges
// the warps' winners; the row (n if none) is returned on thread 0 only.
template <typename TW, int NT>
__device__ __forceinline__ int pivot_search(const TW* panel, int ldp, int jj, int n, const unsigned char* used,
                                            typename AbsKey<TW>::T* red_k, int* red_i) {
  using KeyT = typename AbsKey<TW>::T;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  KeyT bk = 0;
  int bi = n;
  for (int i = tid; i < n; i += NT) {
    if (used[i]) continue;
    key_merge(bk, bi, AbsKey<TW>::of(panel[i * ldp + jj]), i);
  }
  warp_key_max(bk, bi);
  if (lane == 0) {
    red_k[warp] = bk;
    red_i[warp] = bi;
  }
  __syncthreads();
  if (warp == 0) {
    bk = lane < NT / 32 ? red_k[lane] : KeyT(0);
    bi = lane < NT / 32 ? red_i[lane] : n;
    warp_key_max(bk, bi);
  }
  return bi;
}

// log|det| = sum_k log|pivot_k| by warp 0: one log per lane at a time, then a warp tree
// (the result is valid on thread 0).
__device__ __forceinline__ double sum_log_pivots(const double* pabs, int n, bool skip) {
  const int lane = threadIdx.x & 31;
  double part = 0.0;
  if (!skip)
    for (int k = lane; k < n; k += 32) part += log(pabs[k]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
  return part;
}

// TW: working precision; TOUT: inverse output precision.
// TH threads per CTA (one matrix): 1024 hides the DFMA latency inside one CTA; the
// determinant-only path runs 256-thread CTAs with 8-column panels, several per SM, so that
// one matrix's serial pivot steps overlap the trailing updates of the others (measured on
// 1024 matrices of 224: W 8 / 256 threads 1.8x faster than W 16 / 1024 threads).
//
// The FP64 pipe of sm_103a issues one warp-wide DFMA per SM sub-partition about every 64
// cycles, so the serial part of a pivot step (search, reciprocal, log) is kept off it: the
// search compares integer keys, one thread takes the reciprocal and shares it, and the logs
// of the pivots are summed by all threads at the end.
template <typename TW, typename TOUT, bool kInverse, int W, int TH = kThreads>
__global__ void __launch_bounds__(TH) k_gj(TW* __restrict__ mats, int n, const int32_t* __restrict__ list,
                                                 TOUT* __restrict__ binv, double* __restrict__ logabs_out,
                                                 int32_t* __restrict__ sign_out, int32_t* __restrict__ status) {
  static_assert((W & (W - 1)) == 0, "the panel width is a power of two");
  extern __shared__ unsigned char smem_raw[];
  using KeyT = typename AbsKey<TW>::T;
  double* pabs = reinterpret_cast<double*>(smem_raw);  // [n] |pivot| of column k (log taken at the end)
  TW* panel = reinterpret_cast<TW*>(pabs + n);         // [n][W]
  TW* prow = panel + (size_t)n * W;              // [W][n]
  TW* colk = prow + (size_t)W * n;               // [n]
  TW* rowp = colk + n;                           // [W]
  int* piv = reinterpret_cast<int*>(rowp + W);   // [n] pivot row of column k
  int* qinv = piv + n;                           // [n] column whose pivot row is r
  unsigned char* used = reinterpret_cast<unsigned char*>(qinv + n);  // [n]
  __shared__ KeyT red_k[TH / 32];
  __shared__ int red_i[TH / 32];
  __shared__ TW s_inv;
  __shared__ int s_p;
  __shared__ int s_singular;

  const int b = list ? list[blockIdx.x] : blockIdx.x;
  if (b < 0) return;
  TW* A = mats + (size_t)b * n * n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int i = tid; i < n; i += TH) used[i] = 0;
  if (tid == 0) s_singular = 0;
  int sgn = 1;  // kept by thread 0
  __syncthreads();

  for (int K0 = 0; K0 < n; K0 += W) {
    const int w = min(W, n - K0);
    // panel <- columns [K0, K0+w)
    for (int q = tid; q < n * W; q += TH) {
      const int i = q / W, j = q % W;
      if (j < w) panel[q] = A[(size_t)i * n + K0 + j];
    }
    __syncthreads();
    for (int jj = 0; jj < w; ++jj) {
      const int k = K0 + jj;
      const int bi = pivot_search<TW, TH>(panel, W, jj, n, used, red_k, red_i);
      if (tid == 0) {
        if (bi >= n || !(fabs(panel[bi * W + jj]) > TW(0))) {
          s_singular = 1;
        } else {
          const TW pv = panel[bi * W + jj];
          s_inv = TW(1) / pv;
          s_p = bi;
          piv[k] = bi;
          used[bi] = 1;
          pabs[k] = fabs((double)pv);
          if (pv < TW(0)) sgn = -sgn;
        }
      }
      __syncthreads();
      if (s_singular) break;
      const int p = s_p;
      const TW inv = s_inv;
      // snapshot the pivot row (panel part) and column jj before updating
      for (int j = tid; j < w; j += TH) rowp[j] = (j == jj) ? inv : panel[p * W + j] * inv;
      for (int i = tid; i < n; i += TH) colk[i] = panel[i * W + jj];
      __syncthreads();
      for (int q = tid; q < n * W; q += TH) {
        const int i = q / W, j = q % W;
        if (j >= w) continue;
        if (i == p) {
          panel[q] = rowp[j];
        } else if (kInverse || !used[i]) {
          const TW f = colk[i];
          const TW base = (j == jj) ? TW(0) : panel[q];
          panel[q] = base - f * rowp[j];
        }
      }
      __syncthreads();
    }
    if (s_singular) break;
    // old pivot rows of the block (all columns outside the panel)
    for (int q = tid; q < w * n; q += TH) {
      const int j = q / n, c = q - j * n;
      prow[j * n + c] = A[(size_t)piv[K0 + j] * n + c];
    }
    __syncthreads();
    // rank-w update of the columns outside the panel: warp per row, lanes over columns,
    // the row's multipliers u_j = U[i][j] in registers
    const int c_lo = kInverse ? 0 : K0 + w;
    for (int i = warp; i < n; i += TH / 32) {
      if (!kInverse && used[i]) continue;
      TW u[W];
#pragma unroll
      for (int j = 0; j < W; ++j) u[j] = (j < w) ? panel[i * W + j] - ((piv[K0 + j] == i) ? TW(1) : TW(0)) : TW(0);
      TW* Ai = A + (size_t)i * n;
      if constexpr (!kInverse) {
        // determinant only: every column from c_lo on lies right of the panel; one column
        // per lane, so a strip wastes at most 31 lanes
        for (int c = c_lo + lane; c < n; c += 32) {
          TW a1 = Ai[c];
#pragma unroll
          for (int j = 0; j < W; ++j)
            if (j < w) a1 += u[j] * prow[j * n + c];
          Ai[c] = a1;
        }
        continue;
      }
      // inverse: every column; two columns per lane in flight while both lie inside the
      // row, then the odd strip alone (no strip runs with its lanes idle); the panel
      // columns are written back from the panel below
      int c = lane;
      for (; c + 32 < n; c += 64) {
        const int c2 = c + 32;
        const bool in1 = !(c >= K0 && c < K0 + w);
        const bool in2 = !(c2 >= K0 && c2 < K0 + w);
        TW a1 = in1 ? Ai[c] : TW(0);
        TW a2 = in2 ? Ai[c2] : TW(0);
#pragma unroll
        for (int j = 0; j < W; ++j) {
          if (j < w) {
            a1 += u[j] * prow[j * n + c];
            a2 += u[j] * prow[j * n + c2];
          }
        }
        if (in1) Ai[c] = a1;
        if (in2) Ai[c2] = a2;
      }
      if (c < n && !(c >= K0 && c < K0 + w)) {
        TW a1 = Ai[c];
#pragma unroll
        for (int j = 0; j < W; ++j)
          if (j < w) a1 += u[j] * prow[j * n + c];
        Ai[c] = a1;
      }
    }
    // write the swept panel back
    for (int q = tid; q < n * W; q += TH) {
      const int i = q / W, j = q % W;
      if (j < w) A[(size_t)i * n + K0 + j] = panel[q];
    }
    __syncthreads();
  }

  const double logdet = warp == 0 ? sum_log_pivots(pabs, n, s_singular != 0) : 0.0;  // on thread 0
  if (tid == 0) {
    int st = 0;
    double la = logdet;
    int sg = sgn;
    if (s_singular) {
      st = SCALE_SAMPLE_SINGULAR;
      la = -INFINITY;
      sg = 0;
    } else {
      // sign of the permutation k -> piv[k]
      for (int k = 0; k < n; ++k) qinv[k] = 0;
      int parity = 0;
      for (int k = 0; k < n; ++k) {
        if (qinv[k]) continue;
        int j = k, len = 0;
        while (!qinv[j]) {
          qinv[j] = 1;
          j = piv[j];
          ++len;
        }
        parity += len - 1;
      }
      if (parity & 1) sg = -sg;
    }
    if (logabs_out) logabs_out[b] = la;
    if (sign_out) sign_out[b] = sg;
    if (status && st) status[b] |= st;
  }
  if (!kInverse) return;
  __syncthreads();
  if (s_singular) {
    if (binv)
      for (int q = tid; q < n * n; q += TH) binv[(size_t)b * n * n + q] = TOUT(0);
    return;
  }
  for (int k = tid; k < n; k += TH) qinv[piv[k]] = k;
  __syncthreads();
  // Binv[s][cf] = A^-1[cf][s] = A_final[piv[cf]][qinv[s]]
  for (int q = tid; q < n * n; q += TH) {
    const int s = q / n, cf = q - s * n;
    binv[(size_t)b * n * n + q] = (TOUT)A[(size_t)piv[cf] * n + qinv[s]];
  }
}

// Inverse mode split over a thread-block cluster of C CTAs per matrix (FP64 working
// precision). The columns are cut into C contiguous ranges of whole W-column blocks; CTA q
// owns its range, and only it reads or writes those columns of A. For each block the owner
// sweeps the W-column panel in its shared memory exactly as k_gj does; after one cluster
// barrier every CTA copies the swept panel and the block's pivot rows from the owner's
// shared memory (distributed shared memory) and applies the rank-W update to its own
// columns. The panel alternates between two buffers, so the owner of the next block can
// sweep while the others still copy: one cluster barrier per block. Every element sees the
// same operations in the same order as in k_gj, so the two kernels give the same bits; the
// cluster version spreads the O(n^3) FP64 update of one matrix over C SMs, which shortens
// the refresh of a large matrix (the serial panel steps stay on one SM).
template <typename TOUT, int W, int C>
__global__ void __launch_bounds__(kThreads) k_gj_cluster(double* __restrict__ mats, int n,
                                                         const int32_t* __restrict__ list, TOUT* __restrict__ binv,
                                                         double* __restrict__ logabs_out, int32_t* __restrict__ sign_out,
                                                         int32_t* __restrict__ status) {
  extern __shared__ unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int q = (int)cluster.block_rank();
  const int mat = blockIdx.x / C;
  const int b = list ? list[mat] : mat;
  if (b < 0) return;  // the whole cluster shares mat, so it leaves together
  double* A = mats + (size_t)b * n * n;
  const int nblocks = (n + W - 1) / W;
  const int bpc = (nblocks + C - 1) / C;  // blocks per CTA
  const int c_lo = min(n, q * bpc * W), c_hi = min(n, (q + 1) * bpc * W);
  const int ncol = c_hi - c_lo, ldp = bpc * W;
  double* pabs = reinterpret_cast<double*>(smem_raw);    // [n] |pivot| of the columns this CTA owns
  double* panels = pabs + n;                             // [2][n][W]
  double* prow = panels + (size_t)2 * n * W;             // [W][ldp]
  double* colk = prow + (size_t)W * ldp;                 // [n]
  double* rowp = colk + n;                               // [W]
  int* piv = reinterpret_cast<int*>(rowp + W);           // [n]
  int* qinv = piv + n;                                   // [n]
  unsigned char* used = reinterpret_cast<unsigned char*>(qinv + n);  // [n]
  __shared__ unsigned long long red_k[kThreads / 32];
  __shared__ int red_i[kThreads / 32];
  __shared__ double s_inv;
  __shared__ int s_p;
  __shared__ int s_singular;
  __shared__ int s_sgn;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < n; i += kThreads) used[i] = 0;
  if (tid == 0) {
    s_singular = 0;
    s_sgn = 1;
  }
  __syncthreads();
  cluster.sync();  // every CTA of the cluster runs before any reads another's shared memory

  bool singular = false;
  for (int blk = 0; blk < nblocks; ++blk) {
    const int K0 = blk * W, w = min(W, n - K0);
    const int owner = blk / bpc;
    double* panel = panels + (size_t)(blk & 1) * n * W;
    if (q == owner) {
      for (int e = tid; e < n * W; e += kThreads) {
        const int i = e / W, j = e % W;
        if (j < w) panel[e] = A[(size_t)i * n + K0 + j];
      }
      __syncthreads();
      for (int jj = 0; jj < w; ++jj) {
        const int k = K0 + jj;
        const int bi = pivot_search<double, kThreads>(panel, W, jj, n, used, red_k, red_i);
        if (tid == 0) {
          if (bi >= n || !(fabs(panel[bi * W + jj]) > 0.0)) {
            s_singular = 1;
          } else {
            const double pv = panel[bi * W + jj];
            s_inv = 1.0 / pv;
            s_p = bi;
            piv[k] = bi;
            used[bi] = 1;
            pabs[k] = fabs(pv);
            if (pv < 0.0) s_sgn = -s_sgn;
          }
        }
        __syncthreads();
        if (s_singular) break;
        const int p = s_p;
        const double inv = s_inv;
        for (int j = tid; j < w; j += kThreads) rowp[j] = (j == jj) ? inv : panel[p * W + j] * inv;
        for (int i = tid; i < n; i += kThreads) colk[i] = panel[i * W + jj];
        __syncthreads();
        for (int e = tid; e < n * W; e += kThreads) {
          const int i = e / W, j = e % W;
          if (j >= w) continue;
          if (i == p) {
            panel[e] = rowp[j];
          } else {
            const double f = colk[i];
            const double base = (j == jj) ? 0.0 : panel[e];
            panel[e] = base - f * rowp[j];
          }
        }
        __syncthreads();
      }
    }
    cluster.sync();  // the owner's swept panel, pivots and singular flag are visible
    const int* o_sing = cluster.map_shared_rank(&s_singular, owner);
    if (*o_sing) {
      singular = true;
      break;
    }
    if (q != owner) {
      const double* o_panel = cluster.map_shared_rank(panel, owner);
      const int* o_piv = cluster.map_shared_rank(piv, owner);
      for (int e = tid; e < n * W; e += kThreads)
        if (e % W < w) panel[e] = o_panel[e];
      for (int j = tid; j < w; j += kThreads) piv[K0 + j] = o_piv[K0 + j];
      __syncthreads();
      for (int j = tid; j < w; j += kThreads) used[piv[K0 + j]] = 1;
    }
    // old pivot rows of the block on this CTA's columns (outside the panel)
    for (int e = tid; e < w * ncol; e += kThreads) {
      const int j = e / ncol, cc = e - j * ncol;
      prow[j * ldp + cc] = A[(size_t)piv[K0 + j] * n + c_lo + cc];
    }
    __syncthreads();
    // rank-w update of this CTA's columns outside the panel (the order of k_gj)
    for (int i = warp; i < n; i += kThreads / 32) {
      double u[W];
#pragma unroll
      for (int j = 0; j < W; ++j) u[j] = (j < w) ? panel[i * W + j] - ((piv[K0 + j] == i) ? 1.0 : 0.0) : 0.0;
      double* Ai = A + (size_t)i * n;
      int c = c_lo + lane;
      for (; c + 32 < c_hi; c += 64) {
        const int c2 = c + 32;
        const bool in1 = !(c >= K0 && c < K0 + w);
        const bool in2 = !(c2 >= K0 && c2 < K0 + w);
        double a1 = in1 ? Ai[c] : 0.0;
        double a2 = in2 ? Ai[c2] : 0.0;
#pragma unroll
        for (int j = 0; j < W; ++j) {
          if (j < w) {
            a1 += u[j] * prow[j * ldp + (c - c_lo)];
            a2 += u[j] * prow[j * ldp + (c2 - c_lo)];
          }
        }
        if (in1) Ai[c] = a1;
        if (in2) Ai[c2] = a2;
      }
      if (c < c_hi && !(c >= K0 && c < K0 + w)) {
        double a1 = Ai[c];
#pragma unroll
        for (int j = 0; j < W; ++j)
          if (j < w) a1 += u[j] * prow[j * ldp + (c - c_lo)];
        Ai[c] = a1;
      }
    }
    if (q == owner) {
      for (int e = tid; e < n * W; e += kThreads) {
        const int i = e / W, j = e % W;
        if (j < w) A[(size_t)i * n + K0 + j] = panel[e];
      }
    }
    __syncthreads();
  }
  cluster.sync();  // all pivots and flags final: rank 0 gathers the pivots of every block
  if (q == 0) {
    // each column's pivot from the CTA that owns its block, summed as in k_gj
    if (!singular)
      for (int k = tid; k < n; k += kThreads) pabs[k] = cluster.map_shared_rank(pabs, (k / W) / bpc)[k];
    __syncthreads();
    const double logdet = warp == 0 ? sum_log_pivots(pabs, n, singular) : 0.0;
    if (tid == 0) {
      double la = logdet;
      int sg = 1;
      for (int r = 0; r < C; ++r) sg *= *cluster.map_shared_rank(&s_sgn, r);
      if (singular) {
        la = -INFINITY;
        sg = 0;
        if (status) status[b] |= SCALE_SAMPLE_SINGULAR;
      } else {
        for (int k = 0; k < n; ++k) qinv[k] = 0;
        int parity = 0;
        for (int k = 0; k < n; ++k) {
          if (qinv[k]) continue;
          int j = k, len = 0;
          while (!qinv[j]) {
            qinv[j] = 1;
            j = piv[j];
            ++len;
          }
          parity += len - 1;
        }
        if (parity & 1) sg = -sg;
      }
      if (logabs_out) logabs_out[b] = la;
      if (sign_out) sign_out[b] = sg;
    }
  }
  if (singular) {
    // zero this CTA's share of the rows of Binv
    const int r0 = (int)((long long)n * q / C), r1 = (int)((long long)n * (q + 1) / C);
    for (int e = tid; e < (r1 - r0) * n; e += kThreads) binv[(size_t)b * n * n + (size_t)r0 * n + e] = TOUT(0);
  } else {
    // Binv[s][cf] = A^-1[cf][s] = A_final[piv[cf]][col] with s = piv[col], col in this CTA's range
    for (int e = tid; e < ncol * n; e += kThreads) {
      const int cc = e / n, cf = e - cc * n, col = c_lo + cc;
      binv[(size_t)b * n * n + (size_t)piv[col] * n + cf] = (TOUT)A[(size_t)piv[cf] * n + col];
    }
  }
  cluster.sync();  // rank 0 read the others' pivots and signs
}

template <typename TOUT, int W, int C>
cudaError_t run_gj_cluster(cudaStream_t st, double* mats, int n, int B, const int32_t* list, TOUT* binv, double* la,
                           int32_t* sg, int32_t* status) {
  const int nblocks = (n + W - 1) / W, bpc = (nblocks + C - 1) / C;
  const size_t smem =
      sizeof(double) * ((size_t)n + 2 * n * W + (size_t)W * bpc * W + n + W) + sizeof(int) * 2 * n + n + 16;
  auto kern = k_gj_cluster<TOUT, W, C>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)B * C);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess || clusters < 1) {
    cudaGetLastError();  // clear; the caller falls back to one CTA per matrix
    return cudaErrorNotSupported;
  }
  return cudaLaunchKernelEx(&cfg, kern, mats, n, list, binv, la, sg, status);
}

template <typename TW, typename TOUT, bool kInverse, int W, int TH = kThreads>
cudaError_t run_gj(cudaStream_t st, TW* mats, int n, int B, const int32_t* list, TOUT* binv, double* la,
                   int32_t* sg, int32_t* status) {
  const size_t smem = sizeof(double) * n + sizeof(TW) * ((size_t)2 * n * W + n + W) + sizeof(int) * 2 * n + n + 16;
  auto kern = k_gj<TW, TOUT, kInverse, W, TH>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<B, TH, smem, st>>>(mats, n, list, binv, la, sg, status);
  return cudaGetLastError();
}

}  // namespace

// FP64 inverse (out_fp64: Binv in double, else float) or determinant only, for B matrices
// [B][n][n] stored in Phi (overwritten).
cudaError_t launch_gj(scale_ctx* c, const double* Phi, int n, int B, const int32_t* list, bool inverse,
                      bool out_fp64, void* Binv, double* logabs, int32_t* sign, int32_t* status) {
  double* A = const_cast<double*>(Phi);
  if (B <= 0) return cudaSuccess;
  if (inverse) {
    // A listed refresh (a few samples whose counter came due) of matrices above 448 rows is
    // latency-bound: one such FP64 inverse takes a single SM about 0.2 s, so it is split
    // over an 8-CTA cluster. Loads and smaller matrices keep one CTA per matrix, which has
    // the higher throughput (measured at 224 rows: a 4-CTA cluster inverts one matrix only
    // 1.5x faster, the serial panel steps and per-block barriers dominate).
    if (n > 448 && list) {
      const cudaError_t e =
          out_fp64 ? run_gj_cluster<double, 8, 8>(c->stream, A, n, B, list, (double*)Binv, logabs, sign, status)
                   : run_gj_cluster<float, 8, 8>(c->stream, A, n, B, list, (float*)Binv, logabs, sign, status);
      if (e != cudaErrorNotSupported) return e;
    }
    if (out_fp64) {
      if (n > 448) return run_gj<double, double, true, 8>(c->stream, A, n, B, list, (double*)Binv, logabs, sign, status);
      return run_gj<double, double, true, 16>(c->stream, A, n, B, list, (double*)Binv, logabs, sign, status);
    }
    if (n > 448) return run_gj<double, float, true, 8>(c->stream, A, n, B, list, (float*)Binv, logabs, sign, status);
    return run_gj<double, float, true, 16>(c->stream, A, n, B, list, (float*)Binv, logabs, sign, status);
  }
  if (n > 448) return run_gj<double, double, false, 8, 512>(c->stream, A, n, B, list, (double*)nullptr, logabs, sign, status);
  // several matrices per SM: small CTAs overlap one's pivot steps with the others' updates;
  // fewer matrices than a few per SM: one wide CTA per matrix
  if (B < 4 * 152) return run_gj<double, double, false, 16>(c->stream, A, n, B, list, (double*)nullptr, logabs, sign, status);
  return run_gj<double, double, false, 8, 256>(c->stream, A, n, B, list, (double*)nullptr, logabs, sign, status);
}

}  // namespace scale
