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

template <typename TW>
__device__ __forceinline__ void argmax_merge(TW& v, int& i, TW v2, int i2) {
  if (v2 > v || (v2 == v && i2 < i)) {
    v = v2;
    i = i2;
  }
}

// TW: working precision; TOUT: inverse output precision.
// TH threads per CTA (one matrix): 1024 hides the DFMA latency inside one CTA; the
// determinant-only path runs 256-thread CTAs with 8-column panels, several per SM, so that
// one matrix's serial pivot steps overlap the trailing updates of the others (measured on
// 1024 matrices of 224: W 8 / 256 threads 1.8x faster than W 16 / 1024 threads).
template <typename TW, typename TOUT, bool kInverse, int W, int TH = kThreads>
__global__ void __launch_bounds__(TH) k_gj(TW* __restrict__ mats, int n, const int32_t* __restrict__ list,
                                                 TOUT* __restrict__ binv, double* __restrict__ logabs_out,
                                                 int32_t* __restrict__ sign_out, int32_t* __restrict__ status) {
  extern __shared__ unsigned char smem_raw[];
  using KeyT = typename AbsKey<TW>::T;
  // small determinant-only CTAs (several matrices per SM): integer-key pivot search, log|pivot|
  // summed by all threads at the end, one column per lane; the 1024-thread kernels keep FP
  // compares, the running log and two columns per lane (their registers stay unspilled)
  constexpr bool kLean = !kInverse && TH <= 512;
  double* pabs = reinterpret_cast<double*>(smem_raw);  // [n] |pivot| of column k (log taken at the end)
  TW* panel = reinterpret_cast<TW*>(pabs + n);         // [n][W]
  TW* prow = panel + (size_t)n * W;              // [W][n]
  TW* colk = prow + (size_t)W * n;               // [n]
  TW* rowp = colk + n;                           // [W]
  int* piv = reinterpret_cast<int*>(rowp + W);   // [n] pivot row of column k
  int* qinv = piv + n;                           // [n] column whose pivot row is r
  unsigned char* used = reinterpret_cast<unsigned char*>(qinv + n);  // [n]
  __shared__ KeyT red_k[TH / 32];
  __shared__ TW red_v[TH / 32];
  __shared__ int red_i[TH / 32];
  __shared__ double red_l[TH / 32];
  __shared__ int s_p;
  __shared__ int s_singular;

  const int b = list ? list[blockIdx.x] : blockIdx.x;
  if (b < 0) return;
  TW* A = mats + (size_t)b * n * n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (int i = tid; i < n; i += TH) used[i] = 0;
  if (tid == 0) s_singular = 0;
  double logdet = 0.0;  // inverse mode: kept by thread 0
  int sgn = 1;          // kept by thread 0
  __syncthreads();

  for (int K0 = 0; K0 < n; K0 += W) {
    const int w = min(W, n - K0);
    // panel <- columns [K0, K0+w)
    for (int q = tid; q < n * w; q += TH) {
      const int i = q / w, j = q - i * w;
      panel[i * W + j] = A[(size_t)i * n + K0 + j];
    }
    __syncthreads();
    for (int jj = 0; jj < w; ++jj) {
      const int k = K0 + jj;
      // pivot search over unpivoted rows (largest |value|, ties to the lowest row); the
      // determinant-only kernels compare integer keys, the inverse kernels FP values
      int bi = n;
      if constexpr (kLean) {
        KeyT bk = 0;
        for (int i = tid; i < n; i += TH) {
          if (used[i]) continue;
          key_merge(bk, bi, AbsKey<TW>::of(panel[i * W + jj]), i);
        }
        for (int off = 16; off > 0; off >>= 1) {
          const KeyT k2 = __shfl_down_sync(0xffffffffu, bk, off);
          const int i2 = __shfl_down_sync(0xffffffffu, bi, off);
          key_merge(bk, bi, k2, i2);
        }
        if (lane == 0) red_k[warp] = bk;
      } else {
        TW bv = TW(-1);
        for (int i = tid; i < n; i += TH) {
          if (used[i]) continue;
          argmax_merge(bv, bi, TW(fabs(panel[i * W + jj])), i);
        }
        for (int off = 16; off > 0; off >>= 1) {
          const TW v2 = __shfl_down_sync(0xffffffffu, bv, off);
          const int i2 = __shfl_down_sync(0xffffffffu, bi, off);
          argmax_merge(bv, bi, v2, i2);
        }
        if (lane == 0) red_v[warp] = bv;
      }
      if (lane == 0) red_i[warp] = bi;
      __syncthreads();
      if (tid == 0) {
        int i = red_i[0];
        if constexpr (kLean) {
          KeyT kk = red_k[0];
          for (int q = 1; q < TH / 32; ++q) key_merge(kk, i, red_k[q], red_i[q]);
        } else {
          TW v = red_v[0];
          for (int q = 1; q < TH / 32; ++q) argmax_merge(v, i, red_v[q], red_i[q]);
        }
        if (i >= n || !(fabs(panel[i * W + jj]) > TW(0))) {
          s_singular = 1;
          i = 0;
        }
        s_p = i;
      }
      __syncthreads();
      if (s_singular) break;
      const int p = s_p;
      const TW pv = panel[p * W + jj];
      const TW inv = TW(1) / pv;
      // snapshot the pivot row (panel part) and column jj before updating
      for (int j = tid; j < w; j += TH) rowp[j] = (j == jj) ? inv : panel[p * W + j] * inv;
      for (int i = tid; i < n; i += TH) colk[i] = panel[i * W + jj];
      if (tid == 0) {
        piv[k] = p;
        used[p] = 1;
        if constexpr (!kLean) logdet += log(fabs((double)pv));
        else pabs[k] = fabs((double)pv);
        if (pv < TW(0)) sgn = -sgn;
      }
      __syncthreads();
      for (int q = tid; q < n * w; q += TH) {
        const int i = q / w, j = q - i * w;
        if (i == p) {
          panel[i * W + j] = rowp[j];
        } else if (kInverse || !used[i]) {
          const TW f = colk[i];
          const TW base = (j == jj) ? TW(0) : panel[i * W + j];
          panel[i * W + j] = base - f * rowp[j];
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
    // the row's multipliers u_j = U[i][j] in registers, two columns per lane in flight
    const int c_lo = kInverse ? 0 : K0 + w;
    for (int i = warp; i < n; i += TH / 32) {
      if (!kInverse && used[i]) continue;
      TW u[W];
#pragma unroll
      for (int j = 0; j < W; ++j) u[j] = (j < w) ? panel[i * W + j] - ((piv[K0 + j] == i) ? TW(1) : TW(0)) : TW(0);
      TW* Ai = A + (size_t)i * n;
      if constexpr (kLean) {
        // determinant only: every column from c_lo on lies right of the panel; one column
        // per lane (several matrices per SM supply the parallelism), so a strip wastes at most
        // 31 lanes instead of 63
        for (int c = c_lo + lane; c < n; c += 32) {
          TW a1 = Ai[c];
#pragma unroll
          for (int j = 0; j < W; ++j)
            if (j < w) a1 += u[j] * prow[j * n + c];
          Ai[c] = a1;
        }
        continue;
      }
      for (int c = c_lo + lane; c < n; c += 64) {
        const int c2 = c + 32;
        const bool in1 = !(c >= K0 && c < K0 + w);
        const bool in2 = c2 < n && !(c2 >= K0 && c2 < K0 + w);
        TW a1 = in1 ? Ai[c] : TW(0);
        TW a2 = in2 ? Ai[c2] : TW(0);
#pragma unroll
        for (int j = 0; j < W; ++j) {
          if (j < w) {
            a1 += u[j] * prow[j * n + c];
            if (c2 < n) a2 += u[j] * prow[j * n + c2];
          }
        }
        if (in1) Ai[c] = a1;
        if (in2) Ai[c2] = a2;
      }
    }
    // write the swept panel back
    for (int q = tid; q < n * w; q += TH) {
      const int i = q / w, j = q - i * w;
      A[(size_t)i * n + K0 + j] = panel[i * W + j];
    }
    __syncthreads();
  }

  // determinant only: log|det| = sum of log|pivot|, one log per thread
  if constexpr (kLean) {
    double part = 0.0;
    if (!s_singular)
      for (int k = tid; k < n; k += TH) part += log(pabs[k]);
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    if (lane == 0) red_l[warp] = part;
    __syncthreads();
    if (tid == 0)
      for (int q = 0; q < TH / 32; ++q) logdet += red_l[q];
  }
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
  double* panels = reinterpret_cast<double*>(smem_raw);  // [2][n][W]
  double* prow = panels + (size_t)2 * n * W;             // [W][ldp]
  double* colk = prow + (size_t)W * ldp;                 // [n]
  double* rowp = colk + n;                               // [W]
  int* piv = reinterpret_cast<int*>(rowp + W);           // [n]
  int* qinv = piv + n;                                   // [n]
  unsigned char* used = reinterpret_cast<unsigned char*>(qinv + n);  // [n]
  __shared__ double red_v[kThreads / 32];
  __shared__ int red_i[kThreads / 32];
  __shared__ int s_p;
  __shared__ int s_singular;
  __shared__ double s_logdet;
  __shared__ int s_sgn;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < n; i += kThreads) used[i] = 0;
  if (tid == 0) {
    s_singular = 0;
    s_logdet = 0.0;
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
      // log|det| continues from the previous block's owner, so the pivots are summed in
      // order exactly as in k_gj (that owner no longer changes its total)
      if (tid == 0 && blk > 0 && (blk - 1) / bpc != q) s_logdet = *cluster.map_shared_rank(&s_logdet, (blk - 1) / bpc);
      for (int e = tid; e < n * w; e += kThreads) {
        const int i = e / w, j = e - i * w;
        panel[i * W + j] = A[(size_t)i * n + K0 + j];
      }
      __syncthreads();
      for (int jj = 0; jj < w; ++jj) {
        const int k = K0 + jj;
        double bv = -1.0;
        int bi = n;
        for (int i = tid; i < n; i += kThreads) {
          if (used[i]) continue;
          argmax_merge(bv, bi, fabs(panel[i * W + jj]), i);
        }
        for (int off = 16; off > 0; off >>= 1) {
          const double v2 = __shfl_down_sync(0xffffffffu, bv, off);
          const int i2 = __shfl_down_sync(0xffffffffu, bi, off);
          argmax_merge(bv, bi, v2, i2);
        }
        if (lane == 0) {
          red_v[warp] = bv;
          red_i[warp] = bi;
        }
        __syncthreads();
        if (tid == 0) {
          double v = red_v[0];
          int i = red_i[0];
          for (int r = 1; r < kThreads / 32; ++r) argmax_merge(v, i, red_v[r], red_i[r]);
          if (!(v > 0.0) || i >= n) {
            s_singular = 1;
            i = 0;
          }
          s_p = i;
        }
        __syncthreads();
        if (s_singular) break;
        const int p = s_p;
        const double pv = panel[p * W + jj];
        const double inv = 1.0 / pv;
        for (int j = tid; j < w; j += kThreads) rowp[j] = (j == jj) ? inv : panel[p * W + j] * inv;
        for (int i = tid; i < n; i += kThreads) colk[i] = panel[i * W + jj];
        if (tid == 0) {
          piv[k] = p;
          used[p] = 1;
          s_logdet += log(fabs(pv));
          if (pv < 0.0) s_sgn = -s_sgn;
        }
        __syncthreads();
        for (int e = tid; e < n * w; e += kThreads) {
          const int i = e / w, j = e - i * w;
          if (i == p) {
            panel[i * W + j] = rowp[j];
          } else {
            const double f = colk[i];
            const double base = (j == jj) ? 0.0 : panel[i * W + j];
            panel[i * W + j] = base - f * rowp[j];
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
      for (int e = tid; e < n * w; e += kThreads) {
        const int i = e / w, j = e - i * w;
        panel[i * W + j] = o_panel[i * W + j];
      }
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
      for (int c = c_lo + lane; c < c_hi; c += 64) {
        const int c2 = c + 32;
        const bool in1 = !(c >= K0 && c < K0 + w);
        const bool in2 = c2 < c_hi && !(c2 >= K0 && c2 < K0 + w);
        double a1 = in1 ? Ai[c] : 0.0;
        double a2 = in2 ? Ai[c2] : 0.0;
#pragma unroll
        for (int j = 0; j < W; ++j) {
          if (j < w) {
            a1 += u[j] * prow[j * ldp + (c - c_lo)];
            if (c2 < c_hi) a2 += u[j] * prow[j * ldp + (c2 - c_lo)];
          }
        }
        if (in1) Ai[c] = a1;
        if (in2) Ai[c2] = a2;
      }
    }
    if (q == owner) {
      for (int e = tid; e < n * w; e += kThreads) {
        const int i = e / w, j = e - i * w;
        A[(size_t)i * n + K0 + j] = panel[i * W + j];
      }
    }
    __syncthreads();
  }
  cluster.sync();  // all pivots, determinants and flags final; no CTA reads another after this
  if (q == 0 && tid == 0) {
    double la = *cluster.map_shared_rank(&s_logdet, (nblocks - 1) / bpc);  // the running total
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
  cluster.sync();  // rank 0 read the others' determinants
}

template <typename TOUT, int W, int C>
cudaError_t run_gj_cluster(cudaStream_t st, double* mats, int n, int B, const int32_t* list, TOUT* binv, double* la,
                           int32_t* sg, int32_t* status) {
  const int nblocks = (n + W - 1) / W, bpc = (nblocks + C - 1) / C;
  const size_t smem = sizeof(double) * ((size_t)2 * n * W + (size_t)W * bpc * W + n + W) + sizeof(int) * 2 * n + n + 16;
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
