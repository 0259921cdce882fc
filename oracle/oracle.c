/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the SCALE local-energy path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or load this
 * file; only the tests, the smoke check and the bench's CPU-baseline leg use it. It
 * shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (arXiv 2604.25775, Sec. II):
 *   * the SCALE network: per-site embedding E_i[n_i] (Sec. II.B "Embedding Layer"),
 *     k x k convolution layers with residual (Eq. conv) and site-wise layers (Eq. MLP),
 *     both expressed as a layer with a per-layer kernel size and residual flag,
 *     boundary conditions of the Hamiltonian (circular on periodic axes, zero padding
 *     on open ones);
 *   * the orbital projection (Sec. II.B "Orbital Projection"):
 *       M[(s,i)][k] = M0[(s,i)][k] + proj_b[s*Ne+k] + sum_c H_i[c] proj_w[c][s*Ne+k],
 *     orbital o = s*N + i (s = 0 up, 1 down), Phi = rows of M of occupied orbitals in
 *     ascending orbital order;
 *   * psi = det Phi by LU with partial pivoting (log|det|, sign);
 *   * H acting on the occupation basis by second-quantised algebra with Jordan-Wigner
 *     signs (Eq. H_h, Eq. ham-tj), the t-J model restricted to the Gutzwiller-projected
 *     space;
 *   * E_loc(n) = sum_n' <n|H|n'> psi(n')/psi(n) (Sec. II.A) with EVERY psi(n') from a
 *     full network forward plus a fresh LU (the O(N^4) route of Sec. III.A);
 *   * d log|psi| / d theta by a hand-written FP64 backward pass;
 *   * Metropolis steps n -> n' with acceptance min(1, |psi(n')/psi(n)|^2) (Sec. II.A);
 *   * the symmetry-projected amplitude sum_g Pi(n, g) chi_g psi(g n) (App. "Symmetry
 *     Projection");
 *   * the ACE network (Sec. II "ACE", Eq. ACE): the embedding, then n_conv blocks
 *       H(l+1) = LN( H(l) + SiLU(Conv_l(H(l))) )
 *     with LN the layer normalisation of each site's channel vector (mean and biased
 *     variance over the channels, (x - mean) / sqrt(var + eps) * gamma + beta), then the
 *     site-wise layers of Eq. MLP at width h_mlp and the orbital projection. Every psi
 *     that the functions above take goes through the same amplitude routine, so the ACE
 *     log psi, local energy (full recompute of every psi(n')) and symmetry projection
 *     follow from it;
 *   * the wide SCALE shapes of Table tab:model (family 2): the SCALE layout with per-layer
 *     widths (conv h, site-wise h_mlp) and no normalisation, and the plus-shaped stencil of
 *     SCALE-L (stencil 1: the offsets of a k x k box with dx^2 + dy^2 <= ((k-1)/2)^2, 13
 *     sites for k = 5, weights stored for those taps only, in row-major box order).
 *
 * Parity status: every function here is pinned by CPU tests (closed-form U=0 energy,
 * library convolution and slogdet, dense-Hamiltonian enumeration, finite differences,
 * locality of the receptive field). The t-J exchange sign is pinned only by the
 * enumeration identity on tiny lattices.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_MAX_LAYERS 32

typedef struct {
  int32_t Lx, Ly, pbc_x, pbc_y, n_up, n_dn, model; /* model: 0 Hubbard, 1 t-J, 2 Hubbard after PHT */
  double t, tp, U, J;
  int32_t n_layers, h, act, per_site_embed; /* act: 0 tanh, 1 SiLU */
  int32_t ksize[ORA_MAX_LAYERS];
  int32_t residual[ORA_MAX_LAYERS];
  int32_t family;       /* 0 SCALE, 1 ACE, 2 SCALE at per-layer widths (full recompute) */
  int32_t n_conv;       /* ACE: layers [0, n_conv) are conv blocks with layer normalisation */
  int32_t h_mlp;        /* ACE: width of the site-wise layers after the conv blocks */
  double ln_eps;        /* ACE: epsilon of the layer normalisation */
  int32_t stencil;      /* 0: k x k box; 1: the box offsets within L2 distance (k-1)/2 */
  const double *params; /* flat parameter vector (layout in the Python wrapper) */
  const double *M0;     /* [2N][Ne] reference orbitals */
} ora_model;

/* ------------------------------------------------------------------------------------
 * Lattice helpers. Site i = y*Lx + x.
 * ------------------------------------------------------------------------------------ */

/* Site reached from i by the offset (dx, dy), or -1 when it falls off an open edge. */
static int site_offset(const ora_model *m, int i, int dx, int dy) {
  int x = i % m->Lx + dx, y = i / m->Lx + dy;
  if (x < 0 || x >= m->Lx) {
    if (!m->pbc_x) return -1;
    x = ((x % m->Lx) + m->Lx) % m->Lx;
  }
  if (y < 0 || y >= m->Ly) {
    if (!m->pbc_y) return -1;
    y = ((y % m->Ly) + m->Ly) % m->Ly;
  }
  return y * m->Lx + x;
}

/* Bond list of Eq. H_h: nearest neighbours (i, i+x), (i, i+y) when which == 0, next-nearest
 * (i, i+x+y), (i, i+x-y) when which == 1. Each unordered pair once. Returns the count. */
int ora_bonds(const ora_model *m, int which, int32_t *pairs) {
  int N = m->Lx * m->Ly, nb = 0;
  for (int i = 0; i < N; ++i) {
    int offs[2][2];
    if (which == 0) {
      offs[0][0] = 1; offs[0][1] = 0; offs[1][0] = 0; offs[1][1] = 1;
    } else {
      offs[0][0] = 1; offs[0][1] = 1; offs[1][0] = 1; offs[1][1] = -1;
    }
    for (int d = 0; d < 2; ++d) {
      int j = site_offset(m, i, offs[d][0], offs[d][1]);
      if (j < 0) continue;
      if (pairs) { pairs[2 * nb] = i; pairs[2 * nb + 1] = j; }
      ++nb;
    }
  }
  return nb;
}

/* Channel widths. SCALE: every layer has h channels. ACE: the conv blocks keep h, the
 * site-wise layers after them have h_mlp (the first one maps h -> h_mlp). */
static int width_out(const ora_model *m, int l) {
  return (m->family != 0 && l >= m->n_conv) ? m->h_mlp : m->h;
}
/* Whether the offset (dx, dy) belongs to the stencil of a k x k layer. */
static int in_stencil(const ora_model *m, int k, int dx, int dy) {
  const int r = (k - 1) / 2;
  return m->stencil == 0 || dx * dx + dy * dy <= r * r;
}
static int taps_of(const ora_model *m, int k) {
  int n = 0;
  for (int dy = -(k - 1) / 2; dy <= (k - 1) / 2; ++dy)
    for (int dx = -(k - 1) / 2; dx <= (k - 1) / 2; ++dx) n += in_stencil(m, k, dx, dy);
  return n;
}
static int width_in(const ora_model *m, int l) { return l == 0 ? m->h : width_out(m, l - 1); }
static int width_last(const ora_model *m) { return m->n_layers ? width_out(m, m->n_layers - 1) : m->h; }
static int width_max(const ora_model *m) {
  return (m->family != 0 && m->h_mlp > m->h && m->n_layers > m->n_conv) ? m->h_mlp : m->h;
}
static int has_ln(const ora_model *m, int l) { return m->family == 1 && l < m->n_conv; }

int64_t ora_param_count(const ora_model *m) {
  int64_t N = (int64_t)m->Lx * m->Ly, h = m->h, Ne = m->n_up + m->n_dn;
  int64_t n = (m->per_site_embed ? N : 1) * 4 * h;
  for (int l = 0; l < m->n_layers; ++l) {
    const int64_t ci = width_in(m, l), co = width_out(m, l);
    n += (int64_t)taps_of(m, m->ksize[l]) * ci * co + co;
    if (has_ln(m, l)) n += 2 * co;
  }
  n += (int64_t)width_last(m) * 2 * Ne + 2 * Ne;
  return n;
}

/* Offsets of the parameter tensors inside the flat vector. */
typedef struct {
  int64_t embed, kernel[ORA_MAX_LAYERS], bias[ORA_MAX_LAYERS], ln_g[ORA_MAX_LAYERS], ln_b[ORA_MAX_LAYERS];
  int64_t proj_w, proj_b, total;
} ora_offsets;

/* Layer l: kernel [k][k][c_in][c_out], bias [c_out], then (ACE conv blocks) gamma and beta
 * [c_out] of the layer normalisation; then proj_w [c_last][2Ne], proj_b [2Ne]. */
static ora_offsets offsets_of(const ora_model *m) {
  ora_offsets o;
  int64_t N = (int64_t)m->Lx * m->Ly, h = m->h, Ne = m->n_up + m->n_dn;
  int64_t p = 0;
  o.embed = p; p += (m->per_site_embed ? N : 1) * 4 * h;
  for (int l = 0; l < m->n_layers; ++l) {
    const int64_t ci = width_in(m, l), co = width_out(m, l);
    o.kernel[l] = p; p += (int64_t)taps_of(m, m->ksize[l]) * ci * co;
    o.bias[l] = p; p += co;
    o.ln_g[l] = o.ln_b[l] = -1;
    if (has_ln(m, l)) {
      o.ln_g[l] = p; p += co;
      o.ln_b[l] = p; p += co;
    }
  }
  o.proj_w = p; p += (int64_t)width_last(m) * 2 * Ne;
  o.proj_b = p; p += 2 * Ne;
  o.total = p;
  return o;
}

static double act_f(int act, double z) {
  if (act == 0) return tanh(z);
  return z / (1.0 + exp(-z)); /* SiLU */
}

static double act_df(int act, double z) {
  if (act == 0) {
    double th = tanh(z);
    return 1.0 - th * th;
  }
  double s = 1.0 / (1.0 + exp(-z));
  return s * (1.0 + z * (1.0 - s));
}

/* ------------------------------------------------------------------------------------
 * Network forward (Sec. II.B; ACE blocks of Eq. ACE). H holds L+1 layers of [N][hmax]
 * (row stride hmax = width_max, layer l using its first width entries); Z (optional, SCALE
 * only) holds the pre-activation of every layer [L][N][h].
 *   H0_i = E_i[n_i]
 *   u_i = res_l * H(l)_i + act( b_l + sum_{offset d} sum_c' H(l)_{i+d}[c'] K_l[d][c'][.] )
 *   H(l+1)_i = u_i, or LN(u_i) for an ACE conv block:
 *     mean = sum_c u_i[c] / C, var = sum_c (u_i[c] - mean)^2 / C,
 *     H(l+1)_i[c] = (u_i[c] - mean) / sqrt(var + eps) * gamma_l[c] + beta_l[c].
 * A site-wise layer is the k = 1 case.
 * ------------------------------------------------------------------------------------ */
static void forward(const ora_model *m, const int8_t *occ, double *H, double *Z) {
  const int N = m->Lx * m->Ly, h = m->h, hs = width_max(m);
  const ora_offsets off = offsets_of(m);
  const double *P = m->params;
  for (int i = 0; i < N; ++i) {
    const double *e = P + off.embed + ((m->per_site_embed ? (int64_t)i * 4 : 0) + occ[i]) * h;
    for (int c = 0; c < h; ++c) H[(int64_t)i * hs + c] = e[c];
  }
  for (int l = 0; l < m->n_layers; ++l) {
    const double *in = H + (int64_t)l * N * hs;
    double *out = H + (int64_t)(l + 1) * N * hs;
    const int k = m->ksize[l], r = (k - 1) / 2, ci_n = width_in(m, l), co_n = width_out(m, l);
    const double *K = P + off.kernel[l];
    const double *b = P + off.bias[l];
    for (int i = 0; i < N; ++i) {
      for (int co = 0; co < co_n; ++co) {
        double z = b[co];
        int tap = 0; /* index of the offset among the stencil's taps, row-major over the box */
        for (int ky = 0; ky < k; ++ky)
          for (int kx = 0; kx < k; ++kx) {
            if (!in_stencil(m, k, kx - r, ky - r)) continue;
            const int t = tap++;
            int j = site_offset(m, i, kx - r, ky - r);
            if (j < 0) continue; /* zero padding on open edges */
            const double *w = K + ((int64_t)t * ci_n) * co_n;
            for (int ci = 0; ci < ci_n; ++ci) z += in[(int64_t)j * hs + ci] * w[(int64_t)ci * co_n + co];
          }
        if (Z) Z[((int64_t)l * N + i) * h + co] = z;
        out[(int64_t)i * hs + co] = (m->residual[l] ? in[(int64_t)i * hs + co] : 0.0) + act_f(m->act, z);
      }
      if (has_ln(m, l)) {
        double *u = out + (int64_t)i * hs;
        double mean = 0.0, var = 0.0;
        for (int c = 0; c < co_n; ++c) mean += u[c];
        mean /= co_n;
        for (int c = 0; c < co_n; ++c) var += (u[c] - mean) * (u[c] - mean);
        var /= co_n;
        const double inv = 1.0 / sqrt(var + m->ln_eps);
        const double *g = P + off.ln_g[l], *be = P + off.ln_b[l];
        for (int c = 0; c < co_n; ++c) u[c] = (u[c] - mean) * inv * g[c] + be[c];
      }
    }
  }
}

/* Orbital matrix M [2N][Ne] from the last-layer features (Sec. II.B "Orbital Projection"). */
static void orbitals(const ora_model *m, const double *HL, double *M) {
  const int N = m->Lx * m->Ly, h = width_last(m), hs = width_max(m), Ne = m->n_up + m->n_dn;
  const ora_offsets off = offsets_of(m);
  const double *W = m->params + off.proj_w, *bp = m->params + off.proj_b;
  for (int s = 0; s < 2; ++s)
    for (int i = 0; i < N; ++i) {
      const int o = s * N + i;
      for (int k = 0; k < Ne; ++k) {
        double v = m->M0[(int64_t)o * Ne + k] + bp[s * Ne + k];
        for (int c = 0; c < h; ++c) v += HL[(int64_t)i * hs + c] * W[(int64_t)c * 2 * Ne + s * Ne + k];
        M[(int64_t)o * Ne + k] = v;
      }
    }
}

/* Occupied orbitals of n in ascending order (o = s*N + i); returns their count. */
static int occupied(const ora_model *m, const int8_t *occ, int *orbs) {
  const int N = m->Lx * m->Ly;
  int n = 0;
  for (int s = 0; s < 2; ++s)
    for (int i = 0; i < N; ++i)
      if ((occ[i] >> s) & 1) orbs[n++] = s * N + i;
  return n;
}

/* LU with partial pivoting of the n x n row-major A (destroyed). Returns log|det A| and
 * sets *sign to +1 / -1, or to 0 (with -inf) when a pivot is exactly zero. */
static double lu_slogdet(int n, double *A, int *sign) {
  double logabs = 0.0;
  int sg = 1;
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(A[(int64_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      double v = fabs(A[(int64_t)i * n + k]);
      if (v > best) { best = v; p = i; }
    }
    if (best == 0.0) { *sign = 0; return -INFINITY; }
    if (p != k) {
      for (int j = 0; j < n; ++j) {
        double t = A[(int64_t)k * n + j];
        A[(int64_t)k * n + j] = A[(int64_t)p * n + j];
        A[(int64_t)p * n + j] = t;
      }
      sg = -sg;
    }
    const double piv = A[(int64_t)k * n + k];
    if (piv < 0) sg = -sg;
    logabs += log(fabs(piv));
    for (int i = k + 1; i < n; ++i) {
      const double f = A[(int64_t)i * n + k] / piv;
      A[(int64_t)i * n + k] = f;
      for (int j = k + 1; j < n; ++j) A[(int64_t)i * n + j] -= f * A[(int64_t)k * n + j];
    }
  }
  *sign = sg;
  return logabs;
}

/* Exposed for the library pin against numpy.linalg.slogdet. */
double ora_slogdet(int n, const double *A_in, int32_t *sign) {
  double *A = (double *)malloc(sizeof(double) * n * n);
  memcpy(A, A_in, sizeof(double) * n * n);
  int s;
  double la = lu_slogdet(n, A, &s);
  free(A);
  *sign = s;
  return la;
}

/* Scratch for one amplitude evaluation. */
typedef struct {
  double *H, *M, *Phi;
  int *orbs;
} ora_ws;

static ora_ws ws_alloc(const ora_model *m) {
  const int N = m->Lx * m->Ly, hs = width_max(m), Ne = m->n_up + m->n_dn;
  ora_ws w;
  w.H = (double *)malloc(sizeof(double) * (int64_t)(m->n_layers + 1) * N * hs);
  w.M = (double *)malloc(sizeof(double) * (int64_t)2 * N * Ne);
  w.Phi = (double *)malloc(sizeof(double) * (int64_t)Ne * Ne);
  w.orbs = (int *)malloc(sizeof(int) * 2 * N);
  return w;
}

static void ws_free(ora_ws *w) {
  free(w->H); free(w->M); free(w->Phi); free(w->orbs);
}

static int has_double(const ora_model *m, const int8_t *occ) {
  for (int i = 0; i < m->Lx * m->Ly; ++i)
    if (occ[i] == 3) return 1;
  return 0;
}

/* psi(n) = det Phi(n) (Sec. II.B); Phi rows in ascending orbital order. Returns 0 and
 * sets sign = 0 for configurations outside the model's space (wrong particle numbers, or
 * double occupancy under the Gutzwiller projection of the t-J model). */
static int amplitude(const ora_model *m, const int8_t *occ, ora_ws *w, double *logabs, int *sign) {
  const int N = m->Lx * m->Ly, hs = width_max(m), Ne = m->n_up + m->n_dn;
  int nu = 0, nd = 0;
  for (int i = 0; i < N; ++i) { nu += occ[i] & 1; nd += (occ[i] >> 1) & 1; }
  if (nu != m->n_up || nd != m->n_dn || (m->model == 1 && has_double(m, occ))) {
    *logabs = -INFINITY; *sign = 0;
    return 0;
  }
  forward(m, occ, w->H, NULL);
  orbitals(m, w->H + (int64_t)m->n_layers * N * hs, w->M);
  int n = occupied(m, occ, w->orbs);
  for (int a = 0; a < n; ++a)
    memcpy(w->Phi + (int64_t)a * Ne, w->M + (int64_t)w->orbs[a] * Ne, sizeof(double) * Ne);
  *logabs = lu_slogdet(Ne, w->Phi, sign);
  return 1;
}

int ora_log_psi(const ora_model *m, int B, const int8_t *occ, double *logabs, int32_t *sign) {
  const int N = m->Lx * m->Ly;
#pragma omp parallel
  {
    ora_ws w = ws_alloc(m);
#pragma omp for schedule(dynamic)
    for (int b = 0; b < B; ++b) {
      int s;
      amplitude(m, occ + (int64_t)b * N, &w, &logabs[b], &s);
      sign[b] = s;
    }
    ws_free(&w);
  }
  return 0;
}

/* Features of the last layer [B][N][c_last] and orbital matrices [B][2N][Ne]. */
int ora_orbitals(const ora_model *m, int B, const int8_t *occ, double *HL_out, double *M_out) {
  const int N = m->Lx * m->Ly, h = width_last(m), hs = width_max(m), Ne = m->n_up + m->n_dn;
#pragma omp parallel
  {
    ora_ws w = ws_alloc(m);
#pragma omp for schedule(dynamic)
    for (int b = 0; b < B; ++b) {
      forward(m, occ + (int64_t)b * N, w.H, NULL);
      const double *HL = w.H + (int64_t)m->n_layers * N * hs;
      if (HL_out)
        for (int i = 0; i < N; ++i)
          memcpy(HL_out + ((int64_t)b * N + i) * h, HL + (int64_t)i * hs, sizeof(double) * h);
      if (M_out) orbitals(m, HL, M_out + (int64_t)b * 2 * N * Ne);
    }
    ws_free(&w);
  }
  return 0;
}

/* All layers of the forward pass for one configuration: [(L+1)][N][hmax], layer l in the
 * first entries of each row (hmax = the widest layer). */
int ora_features(const ora_model *m, const int8_t *occ, double *H_out) {
  forward(m, occ, H_out, NULL);
  return 0;
}

/* ------------------------------------------------------------------------------------
 * Hamiltonian action on the occupation basis. Orbital occupation array oo[2N],
 * o = s*N + i. Jordan-Wigner sign of c_o or c+_o on |n> = prod_{o ascending} c+_o |0>:
 * (-1)^(number of occupied orbitals with index < o).
 * ------------------------------------------------------------------------------------ */
static int jw(const int8_t *oo, int o) {
  int c = 0;
  for (int q = 0; q < o; ++q) c += oo[q];
  return (c & 1) ? -1 : 1;
}

static int annihilate(int8_t *oo, int o, int *sg) {
  if (!oo[o]) return 0;
  *sg *= jw(oo, o);
  oo[o] = 0;
  return 1;
}

static int create(int8_t *oo, int o, int *sg) {
  if (oo[o]) return 0;
  *sg *= jw(oo, o);
  oo[o] = 1;
  return 1;
}

static void to_orbitals(int N, const int8_t *occ, int8_t *oo) {
  for (int i = 0; i < N; ++i) { oo[i] = occ[i] & 1; oo[N + i] = (occ[i] >> 1) & 1; }
}

static void from_orbitals(int N, const int8_t *oo, int8_t *occ) {
  for (int i = 0; i < N; ++i) occ[i] = (int8_t)(oo[i] | (oo[N + i] << 1));
}

/* Diagonal part: Hubbard U sum_i n_up n_dn; t-J J sum_<ij> Sz_i Sz_j (Eq. ham-tj carries
 * no -n_i n_j / 4 term); the particle-hole transformed Hubbard model of the attractive-U
 * benchmarks (App. "particle-hole transformation": c_dn -> (-1)^i c_dn^+, so n_dn -> 1 - n_dn)
 * U sum_i n_up (1 - n_dn). */
double ora_diag(const ora_model *m, const int8_t *occ) {
  const int N = m->Lx * m->Ly;
  if (m->model == 0) {
    int d = 0;
    for (int i = 0; i < N; ++i) d += (occ[i] == 3);
    return m->U * d;
  }
  if (m->model == 2) {
    int d = 0;
    for (int i = 0; i < N; ++i) d += (occ[i] & 1) * (1 - ((occ[i] >> 1) & 1));
    return m->U * d;
  }
  int32_t *pr = (int32_t *)malloc(sizeof(int32_t) * 4 * N);
  int nb = ora_bonds(m, 0, pr);
  double e = 0.0;
  for (int b = 0; b < nb; ++b) {
    int i = pr[2 * b], j = pr[2 * b + 1];
    double szi = 0.5 * ((occ[i] & 1) - ((occ[i] >> 1) & 1));
    double szj = 0.5 * ((occ[j] & 1) - ((occ[j] >> 1) & 1));
    e += m->J * szi * szj;
  }
  free(pr);
  return e;
}

/* Off-diagonal connected configurations n' of n with coefficients <n'|H|n>.
 * Writes at most cap entries; returns the number found (may exceed cap). */
int ora_connected(const ora_model *m, const int8_t *occ, int cap, int8_t *xp, double *coeff) {
  const int N = m->Lx * m->Ly;
  int8_t *oo = (int8_t *)malloc(2 * N), *o2 = (int8_t *)malloc(2 * N);
  int8_t *tmp = (int8_t *)malloc(N);
  int32_t *pr = (int32_t *)malloc(sizeof(int32_t) * 4 * N);
  int count = 0;
  to_orbitals(N, occ, oo);
  for (int which = 0; which < 2; ++which) {
    const double tb = which == 0 ? m->t : m->tp;
    if (tb == 0.0) continue;
    int nb = ora_bonds(m, which, pr);
    for (int b = 0; b < nb; ++b)
      for (int s = 0; s < 2; ++s)
        for (int dir = 0; dir < 2; ++dir) {
          int from = dir ? pr[2 * b] : pr[2 * b + 1];
          int to = dir ? pr[2 * b + 1] : pr[2 * b];
          memcpy(o2, oo, 2 * N);
          int sg = 1;
          /* -t c+_{to,s} c_{from,s} */
          if (!annihilate(o2, s * N + from, &sg)) continue;
          if (!create(o2, s * N + to, &sg)) continue;
          from_orbitals(N, o2, tmp);
          if (m->model == 1 && tmp[to] == 3) continue; /* Gutzwiller projection */
          if (count < cap) {
            memcpy(xp + (int64_t)count * N, tmp, N);
            coeff[count] = -tb * sg;
          }
          ++count;
        }
  }
  if (m->model == 1 && m->J != 0.0) {
    int nb = ora_bonds(m, 0, pr);
    for (int b = 0; b < nb; ++b)
      for (int dir = 0; dir < 2; ++dir) {
        int i = dir ? pr[2 * b + 1] : pr[2 * b], j = dir ? pr[2 * b] : pr[2 * b + 1];
        /* (J/2) S+_i S-_j with S+_i = c+_{i up} c_{i dn}, S-_j = c+_{j dn} c_{j up};
         * operators applied right to left. */
        memcpy(o2, oo, 2 * N);
        int sg = 1;
        if (!annihilate(o2, 0 * N + j, &sg)) continue;
        if (!create(o2, 1 * N + j, &sg)) continue;
        if (!annihilate(o2, 1 * N + i, &sg)) continue;
        if (!create(o2, 0 * N + i, &sg)) continue;
        from_orbitals(N, o2, tmp);
        if (count < cap) {
          memcpy(xp + (int64_t)count * N, tmp, N);
          coeff[count] = 0.5 * m->J * sg;
        }
        ++count;
      }
  }
  free(oo); free(o2); free(tmp); free(pr);
  return count;
}

/* E_loc(n) = diag(n) + sum_n' <n'|H|n> psi(n')/psi(n), every psi(n') by full recompute.
 * status[b] = 0 ok, 1 psi(n) = 0 or n outside the model's space (E_loc = NaN). */
int ora_local_energy(const ora_model *m, int B, const int8_t *occ, double *eloc, int32_t *status) {
  const int N = m->Lx * m->Ly;
  const int cap = 12 * N + 8;
#pragma omp parallel
  {
    ora_ws w = ws_alloc(m);
    int8_t *xp = (int8_t *)malloc((int64_t)cap * N);
    double *cf = (double *)malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic)
    for (int b = 0; b < B; ++b) {
      const int8_t *x = occ + (int64_t)b * N;
      double la;
      int sg;
      amplitude(m, x, &w, &la, &sg);
      if (sg == 0) {
        eloc[b] = NAN;
        if (status) status[b] = 1;
        continue;
      }
      double e = ora_diag(m, x);
      int nc = ora_connected(m, x, cap, xp, cf);
      for (int c = 0; c < nc; ++c) {
        double la2;
        int sg2;
        amplitude(m, xp + (int64_t)c * N, &w, &la2, &sg2);
        if (sg2 == 0) continue;
        e += cf[c] * (double)(sg2 * sg) * exp(la2 - la);
      }
      eloc[b] = e;
      if (status) status[b] = 0;
    }
    free(xp); free(cf);
    ws_free(&w);
  }
  return 0;
}

/* psi(n')/psi(n) for one move per sample, moves[b] = (kind, src, dst, spin):
 * kind 0 = hop of spin `spin` from src to dst, kind 1 = exchange of the two sites'
 * single spins, kind -1 = none (ratio 1). Ratio 0 when the move leaves the space. */
int ora_ratio(const ora_model *m, int B, const int8_t *occ, const int32_t *moves, double *ratio) {
  const int N = m->Lx * m->Ly;
#pragma omp parallel
  {
    ora_ws w = ws_alloc(m);
    int8_t *x2 = (int8_t *)malloc(N);
#pragma omp for schedule(dynamic)
    for (int b = 0; b < B; ++b) {
      const int8_t *x = occ + (int64_t)b * N;
      const int32_t *mv = moves + 4 * (int64_t)b;
      if (mv[0] < 0) { ratio[b] = 1.0; continue; }
      memcpy(x2, x, N);
      if (mv[0] == 0) {
        x2[mv[1]] &= (int8_t)~(1 << mv[3]);
        x2[mv[2]] |= (int8_t)(1 << mv[3]);
      } else {
        int8_t t = x2[mv[1]]; x2[mv[1]] = x2[mv[2]]; x2[mv[2]] = t;
      }
      double la, la2;
      int sg, sg2;
      amplitude(m, x, &w, &la, &sg);
      amplitude(m, x2, &w, &la2, &sg2);
      ratio[b] = (sg == 0 || sg2 == 0) ? 0.0 : (double)(sg * sg2) * exp(la2 - la);
    }
    free(x2);
    ws_free(&w);
  }
  return 0;
}

/* ------------------------------------------------------------------------------------
 * Symmetry-projected amplitude (App. "Symmetry Projection"):
 *   psi_sym(n) = sum_g Pi(n, g) chi_g psi(g n).
 * Each group element is an orbital permutation perm[g][o] (o = s*N + i; a lattice symmetry
 * moves the site of both spins, spin inversion exchanges s); g n occupies perm[g][o] for
 * every orbital o occupied in n. Pi(n, g) is the fermionic sign of that relabelling: with
 * o_1 < ... < o_Ne the occupied orbitals of n, the parity of the permutation that sorts
 * (perm[g][o_1], ..., perm[g][o_Ne]) ascending. The characters chi_g are real (one-
 * dimensional real representations, e.g. the fully symmetric one). A g n outside the
 * model's space (wrong particle numbers, double occupancy in t-J) has psi = 0. The sum is
 * accumulated in FP64 as s * exp(m) (largest log|psi| first) and returned as log|psi_sym|
 * and its sign (0 for a vanishing sum).
 * ------------------------------------------------------------------------------------ */
int ora_log_psi_sym(const ora_model *m, int B, const int8_t *occ, int G, const int32_t *perm, const double *chi,
                    double *logabs, int32_t *sign) {
  const int N = m->Lx * m->Ly;
#pragma omp parallel
  {
    ora_ws w = ws_alloc(m);
    int8_t *x2 = (int8_t *)malloc(N);
    int *orbs = (int *)malloc(sizeof(int) * 2 * N);
    int *img = (int *)malloc(sizeof(int) * 2 * N);
#pragma omp for schedule(dynamic)
    for (int b = 0; b < B; ++b) {
      const int8_t *x = occ + (int64_t)b * N;
      const int n = occupied(m, x, orbs);
      double mx = -INFINITY, s = 0.0;
      for (int g = 0; g < G; ++g) {
        const int32_t *pg = perm + (int64_t)g * 2 * N;
        memset(x2, 0, N);
        for (int a = 0; a < n; ++a) {
          img[a] = pg[orbs[a]];
          x2[img[a] % N] |= (int8_t)(1 << (img[a] / N));
        }
        int inv = 0;
        for (int a = 0; a < n; ++a)
          for (int c = a + 1; c < n; ++c) inv += img[a] > img[c];
        double la;
        int sg;
        amplitude(m, x2, &w, &la, &sg);
        if (sg == 0) continue;
        const double c = chi[g] * ((inv & 1) ? -1.0 : 1.0) * sg;
        if (c == 0.0) continue;
        if (la > mx) {
          s = s * exp(mx - la) + c;
          mx = la;
        } else {
          s += c * exp(la - mx);
        }
      }
      logabs[b] = (s == 0.0) ? -INFINITY : mx + log(fabs(s));
      sign[b] = s > 0.0 ? 1 : (s < 0.0 ? -1 : 0);
    }
    free(img);
    free(orbs);
    free(x2);
    ws_free(&w);
  }
  return 0;
}

/* ------------------------------------------------------------------------------------
 * Metropolis sampling of P(n) ~ |psi(n)|^2 by local updates (Sec. II.A; the optimisation
 * settings give 2.5 N steps per sample). The paper does not spell out the proposal; this
 * is the symmetric single-electron hop:
 *   electron  = the pick-th occupied orbital in ascending orbital order (o = s*N + i),
 *   direction = +x, -x, +y, -y for dir = 0..3 (nearest neighbour of its site);
 *   a target off an open edge, or already holding an electron of that spin (t-J: any
 *   electron), is rejected; otherwise the move is accepted when u < |psi(n')/psi(n)|^2.
 * A current amplitude of zero accepts any move to a non-zero amplitude. Every random
 * number is an input: pick [S][B] in [0, Ne), dir [S][B] in [0, 4), u [S][B] in [0, 1).
 * occ [B][N] is advanced in place; accepted[b] counts the accepted steps.
 * ------------------------------------------------------------------------------------ */
int ora_metropolis(const ora_model *m, int B, int S, int8_t *occ, const int32_t *pick, const int32_t *dir,
                   const double *u, int32_t *accepted) {
  const int N = m->Lx * m->Ly, Ne = m->n_up + m->n_dn;
#pragma omp parallel
  {
    ora_ws w = ws_alloc(m);
    int8_t *x2 = (int8_t *)malloc(N);
#pragma omp for schedule(dynamic)
    for (int b = 0; b < B; ++b) {
      int8_t *x = occ + (int64_t)b * N;
      double la;
      int sg;
      amplitude(m, x, &w, &la, &sg);
      accepted[b] = 0;
      for (int st = 0; st < S; ++st) {
        const int64_t q = (int64_t)st * B + b;
        /* the pick-th occupied orbital, ascending */
        int k = pick[q], o_src = -1;
        if (k < 0 || k >= Ne) continue;
        for (int o = 0; o < 2 * N; ++o)
          if ((x[o % N] >> (o / N)) & 1) {
            if (k == 0) { o_src = o; break; }
            --k;
          }
        const int s = o_src / N, i = o_src % N;
        static const int dx[4] = {1, -1, 0, 0}, dy[4] = {0, 0, 1, -1};
        if (dir[q] < 0 || dir[q] > 3) continue;
        const int j = site_offset(m, i, dx[dir[q]], dy[dir[q]]);
        if (j < 0) continue;
        if (m->model == 1 ? x[j] != 0 : ((x[j] >> s) & 1)) continue;
        memcpy(x2, x, N);
        x2[i] &= (int8_t)~(1 << s);
        x2[j] |= (int8_t)(1 << s);
        double la2;
        int sg2;
        amplitude(m, x2, &w, &la2, &sg2);
        int acc;
        if (sg2 == 0) acc = 0;
        else if (sg == 0) acc = 1;
        else acc = u[q] < exp(2.0 * (la2 - la));
        if (acc) {
          memcpy(x, x2, N);
          la = la2;
          sg = sg2;
          accepted[b] += 1;
        }
      }
    }
    free(x2);
    ws_free(&w);
  }
  return 0;
}

/* ------------------------------------------------------------------------------------
 * d log|psi| / d theta, hand-written backward pass.
 *   d log|det Phi| / d Phi[a][k] = (Phi^-1)[k][a]
 *   -> dM rows of occupied orbitals -> proj_w, proj_b, dH^(L)
 *   -> back through every layer (activation derivative, kernel, bias, residual)
 *   -> embedding rows E_i[n_i].
 * grad has the flat parameter layout.
 * ------------------------------------------------------------------------------------ */

/* Inverse of the n x n row-major A by LU with partial pivoting, into Ainv. Returns 0 when
 * singular. */
static int lu_inverse(int n, const double *A, double *Ainv) {
  double *LU = (double *)malloc(sizeof(double) * n * n);
  int *perm = (int *)malloc(sizeof(int) * n);
  memcpy(LU, A, sizeof(double) * n * n);
  for (int i = 0; i < n; ++i) perm[i] = i;
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(LU[(int64_t)k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(LU[(int64_t)i * n + k]) > best) { best = fabs(LU[(int64_t)i * n + k]); p = i; }
    if (best == 0.0) { free(LU); free(perm); return 0; }
    if (p != k) {
      for (int j = 0; j < n; ++j) {
        double t = LU[(int64_t)k * n + j]; LU[(int64_t)k * n + j] = LU[(int64_t)p * n + j]; LU[(int64_t)p * n + j] = t;
      }
      int t = perm[k]; perm[k] = perm[p]; perm[p] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      double f = LU[(int64_t)i * n + k] / LU[(int64_t)k * n + k];
      LU[(int64_t)i * n + k] = f;
      for (int j = k + 1; j < n; ++j) LU[(int64_t)i * n + j] -= f * LU[(int64_t)k * n + j];
    }
  }
  /* Solve A X = I column by column: P A = L U. */
  double *y = (double *)malloc(sizeof(double) * n);
  for (int col = 0; col < n; ++col) {
    for (int i = 0; i < n; ++i) y[i] = (perm[i] == col) ? 1.0 : 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < i; ++j) y[i] -= LU[(int64_t)i * n + j] * y[j];
    for (int i = n - 1; i >= 0; --i) {
      for (int j = i + 1; j < n; ++j) y[i] -= LU[(int64_t)i * n + j] * y[j];
      y[i] /= LU[(int64_t)i * n + i];
    }
    for (int i = 0; i < n; ++i) Ainv[(int64_t)i * n + col] = y[i];
  }
  free(y); free(LU); free(perm);
  return 1;
}

static void grad_one(const ora_model *m, const int8_t *occ, double *g, double *H, double *Z,
                     double *M, double *Phi, double *Pinv, int *orbs, double *dH, double *dZ,
                     double *dIn) {
  const int N = m->Lx * m->Ly, h = m->h, Ne = m->n_up + m->n_dn, L = m->n_layers;
  const ora_offsets off = offsets_of(m);
  const double *P = m->params;
  memset(g, 0, sizeof(double) * off.total);
  forward(m, occ, H, Z);
  const double *HL = H + (int64_t)L * N * h;
  orbitals(m, HL, M);
  int n = occupied(m, occ, orbs);
  for (int a = 0; a < n; ++a) memcpy(Phi + (int64_t)a * Ne, M + (int64_t)orbs[a] * Ne, sizeof(double) * Ne);
  if (!lu_inverse(Ne, Phi, Pinv)) {
    for (int64_t q = 0; q < off.total; ++q) g[q] = NAN;
    return;
  }
  /* dM[o_a][k] = Pinv[k][a]; projection gradients and dH^(L). */
  memset(dH, 0, sizeof(double) * N * h);
  const double *W = P + off.proj_w;
  for (int a = 0; a < n; ++a) {
    const int o = orbs[a], s = o / N, i = o % N;
    for (int k = 0; k < Ne; ++k) {
      const double dm = Pinv[(int64_t)k * Ne + a];
      g[off.proj_b + s * Ne + k] += dm;
      for (int c = 0; c < h; ++c) {
        g[off.proj_w + (int64_t)c * 2 * Ne + s * Ne + k] += HL[(int64_t)i * h + c] * dm;
        dH[(int64_t)i * h + c] += W[(int64_t)c * 2 * Ne + s * Ne + k] * dm;
      }
    }
  }
  /* Back through the layers; dH holds d/dH^(l+1) on entry of step l. */
  for (int l = L - 1; l >= 0; --l) {
    const double *in = H + (int64_t)l * N * h;
    const int k = m->ksize[l], r = (k - 1) / 2;
    const double *K = P + off.kernel[l];
    for (int i = 0; i < N; ++i)
      for (int c = 0; c < h; ++c) {
        const double z = Z[((int64_t)l * N + i) * h + c];
        dZ[(int64_t)i * h + c] = dH[(int64_t)i * h + c] * act_df(m->act, z);
      }
    for (int q = 0; q < N * h; ++q) dIn[q] = m->residual[l] ? dH[q] : 0.0;
    for (int i = 0; i < N; ++i) {
      for (int c = 0; c < h; ++c) g[off.bias[l] + c] += dZ[(int64_t)i * h + c];
      int tap = 0; /* index of the offset among the stencil's taps, row-major over the box */
      for (int ky = 0; ky < k; ++ky)
        for (int kx = 0; kx < k; ++kx) {
          if (!in_stencil(m, k, kx - r, ky - r)) continue;
          const int d = tap++;
          int j = site_offset(m, i, kx - r, ky - r);
          if (j < 0) continue;
          const int64_t wo = off.kernel[l] + (int64_t)d * h * h;
          for (int ci = 0; ci < h; ++ci)
            for (int co = 0; co < h; ++co) {
              g[wo + (int64_t)ci * h + co] += in[(int64_t)j * h + ci] * dZ[(int64_t)i * h + co];
              dIn[(int64_t)j * h + ci] += K[(int64_t)d * h * h + (int64_t)ci * h + co] * dZ[(int64_t)i * h + co];
            }
        }
    }
    memcpy(dH, dIn, sizeof(double) * N * h);
  }
  for (int i = 0; i < N; ++i) {
    const int64_t eo = off.embed + ((m->per_site_embed ? (int64_t)i * 4 : 0) + occ[i]) * h;
    for (int c = 0; c < h; ++c) g[eo + c] += dH[(int64_t)i * h + c];
  }
}

int ora_grad_logpsi(const ora_model *m, int B, const int8_t *occ, double *grad) {
  const int N = m->Lx * m->Ly, h = m->h, Ne = m->n_up + m->n_dn, L = m->n_layers;
  const int64_t P = ora_param_count(m);
  if (m->family != 0) return -1; /* the backward pass covers the SCALE family (either stencil) */
#pragma omp parallel
  {
    double *H = (double *)malloc(sizeof(double) * (int64_t)(L + 1) * N * h);
    double *Z = (double *)malloc(sizeof(double) * (int64_t)L * N * h);
    double *M = (double *)malloc(sizeof(double) * (int64_t)2 * N * Ne);
    double *Phi = (double *)malloc(sizeof(double) * (int64_t)Ne * Ne);
    double *Pinv = (double *)malloc(sizeof(double) * (int64_t)Ne * Ne);
    int *orbs = (int *)malloc(sizeof(int) * 2 * N);
    double *dH = (double *)malloc(sizeof(double) * (int64_t)N * h);
    double *dZ = (double *)malloc(sizeof(double) * (int64_t)N * h);
    double *dIn = (double *)malloc(sizeof(double) * (int64_t)N * h);
#pragma omp for schedule(dynamic)
    for (int b = 0; b < B; ++b)
      grad_one(m, occ + (int64_t)b * N, grad + (int64_t)b * P, H, Z, M, Phi, Pinv, orbs, dH, dZ, dIn);
    free(H); free(Z); free(M); free(Phi); free(Pinv); free(orbs); free(dH); free(dZ); free(dIn);
  }
  return 0;
}

int ora_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
