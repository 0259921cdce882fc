/*
 * scale.h -- C ABI of the GB300 (sm_103a) SCALE local-energy library.
 *
 * The library evaluates, for a batch of lattice-fermion configurations n, the amplitude
 * psi(n) = det Phi(n) of the SCALE convolutional-backflow ansatz (arXiv 2604.25775,
 * Sec. II.B), amplitude ratios psi(n')/psi(n), local energies
 *   E_loc(n) = sum_n' <n|H|n'> psi(n')/psi(n)            (Sec. II.A)
 * for the Hubbard and t-J Hamiltonians (Eq. H_h, Eq. ham-tj), and per-sample gradients
 * d log|psi| / d theta. Ratios use the cached-network + Sherman-Morrison-Woodbury local
 * update of Sec. II.C (Eq. neighbor, Eq. SMW): every connected configuration costs a
 * rank-r determinant det(I_r + V^T Phi^-1 U) against a cached per-sample Phi^-1.
 *
 * Conventions used by every entry point
 *   - Site i = y*Lx + x. Local state n_i in {0 empty, 1 up, 2 down, 3 up+down}, int8.
 *   - Orbital (row of the orbital matrix M) o = s*N + i, s = 0 up, 1 down.
 *   - psi(n) = det of the rows of M of the occupied orbitals in ascending order; log|psi|
 *     and sign are reported in that convention (a global sign of psi is irrelevant to
 *     E_loc and to log-derivatives, this one makes results comparable across codes).
 *   - Parameters: one flat float64 vector, tensors in this order:
 *       embed  [N][4][h] (per_site_embed = 1, tables E_i of Sec. II.B) or [4][h]
 *       for each layer l: kernel [k_l][k_l][h][h] (ky, kx, c_in, c_out), bias [h]
 *         layer l: H(l+1)_i = residual_l * H(l)_i
 *                             + act(bias_l + sum_{|dx|,|dy|<=(k_l-1)/2} H(l)_{i+(dx,dy)} K_l[dy][dx])
 *         (Eq. conv for k_l > 1, Eq. MLP for k_l = 1; offsets wrap on periodic axes and
 *          read zeros past open edges)
 *       proj_w [h][2*Ne], proj_b [2*Ne]: M[(s,i)][k] = M0[(s,i)][k] + proj_b[s*Ne+k]
 *                                             + sum_c H(L)_i[c] proj_w[c][s*Ne+k]
 *     M0 [2N][Ne] float64 is an input (reference orbitals, e.g. plane waves), not a
 *     parameter.
 *   - Moves (connected configurations) are int32 quadruples (kind, src, dst, spin):
 *       kind 0 (hop): the spin-`spin` electron on site src moves to site dst;
 *       kind 1 (exchange, t-J): the single spins on src and dst swap;
 *       kind -1: no move (ratio 1, commit is a no-op).
 *
 * Memory, streams, errors
 *   - Pointer arguments are DEVICE pointers unless the name ends in _host. The caller owns
 *     every pointer it passes; the context owns its cache (features, Phi^-1, projector,
 *     (M0 + proj_b) Phi^-1, slot maps), allocated once at scale_create within the HBM budget.
 *   - Every call is asynchronous on the stream given at creation, except the stated
 *     host-reading calls (scale_get_stats, scale_footprint_bytes). A context is not
 *     re-entrant: one host thread at a time.
 *   - Call-level failures return a scale_status; scale_last_error(ctx) gives the text.
 *     Per-sample problems (wrong particle numbers, double occupancy under the t-J
 *     projection, a singular Phi) never fail the call: the sample's status word is set,
 *     log|psi| = -inf, sign = 0, E_loc = NaN, gradient = NaN.
 */
#ifndef SCALE_H
#define SCALE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SCALE_OK = 0,
  SCALE_EINVAL = 1,       /* bad argument or descriptor */
  SCALE_ENOMEM = 2,       /* device allocation failed */
  SCALE_EBUDGET = 3,      /* request does not fit the HBM budget */
  SCALE_ECUDA = 4,        /* a CUDA call failed (text in scale_last_error) */
  SCALE_ETIMEOUT = 5,     /* a bounded wait ran out */
  SCALE_EUNSUPPORTED = 6, /* valid but not supported by this library (see text) */
  SCALE_ECANCELED = 7     /* a server request was cancelled before it ran */
} scale_status;

/* SCALE_MODEL_HUBBARD_PH: the Hubbard model after the particle-hole transformation of the
 * down spins used for the attractive-U benchmarks (App. "particle-hole transformation",
 * c_dn -> (-1)^i c_dn^+): the same nearest-neighbour hopping and the diagonal
 * U sum_i n_up (1 - n_dn); n_dn counts the transformed down particles (N minus the down
 * electrons of the attractive model). The transformation keeps the hopping form only for
 * nearest-neighbour bonds, so t' must be 0. */
enum { SCALE_MODEL_HUBBARD = 0, SCALE_MODEL_TJ = 1, SCALE_MODEL_HUBBARD_PH = 2 };
enum { SCALE_ACT_TANH = 0, SCALE_ACT_SILU = 1 };
/* Network family. SCALE (Sec. II.B): one k x k residual conv then site-wise layers, all
 * at width h; every entry point. ACE (Sec. II "ACE", Eq. ACE): n_conv residual k x k conv
 * blocks at width h, each followed by a layer normalisation of every site's channel vector
 * (mean and biased variance over the channels, eps = ln_eps, per-channel gain and shift),
 * then site-wise layers at width h_mlp. A local change reaches every site through the
 * stack, so ACE has no cached update: scale_load, scale_log_psi, scale_local_energy with
 * SCALE_PATH_FULL and scale_log_psi_sym run it; the low-rank entry points, the gradient,
 * the server and the allocation-free call return SCALE_EUNSUPPORTED. */
/* SCALE_FAMILY_WIDE: the SCALE layout (one k x k conv, then site-wise layers) at the widths of
 * Table tab:model (conv h up to 1024, site-wise h_mlp up to 2048) and with SCALE-L's
 * plus-shaped stencil. The entry points of ACE apply, and with layer 0 a 3x3 box or a plus
 * of at most 13 sites (n_conv = 1, kernel size 1 after it) also the cached local energies:
 * scale_local_energy with SCALE_PATH_LOWRANK, from a cache (layer-0 pre-activations, the
 * last layer's features, the FP64 inverse and the projector) that scale_load builds. Ratios,
 * commits, sweeps and refreshes are not offered at these shapes (SCALE_EUNSUPPORTED). */
enum { SCALE_FAMILY_SCALE = 0, SCALE_FAMILY_ACE = 1, SCALE_FAMILY_WIDE = 2 };
/* Stencil of the k x k layers: the whole box, or the box offsets within L2 distance
 * (k - 1) / 2 (k = 5: the 13 sites of SCALE-L, Table tab:model); a kernel holds weights for
 * its taps only, [taps][c_in][c_out], taps in row-major box order. */
enum { SCALE_STENCIL_BOX = 0, SCALE_STENCIL_DISK = 1 };
enum { SCALE_PREC_FP64 = 0, SCALE_PREC_MIXED = 1, SCALE_PREC_MIXED_BF16 = 2, SCALE_PREC_MIXED_FP16 = 3 };
enum { SCALE_PATH_LOWRANK = 0, SCALE_PATH_FULL = 1 };

/* per-sample status bits */
enum {
  SCALE_SAMPLE_OK = 0,
  SCALE_SAMPLE_BAD_COUNT = 1,   /* particle numbers differ from n_up / n_dn */
  SCALE_SAMPLE_DOUBLE_OCC = 2,  /* double occupancy in the Gutzwiller-projected t-J space */
  SCALE_SAMPLE_SINGULAR = 4,    /* Phi singular (exact zero pivot) */
  SCALE_SAMPLE_DRIFT = 8        /* drift check fired since the last refresh */
};

#define SCALE_MAX_LAYERS 32

/* Lattice and Hamiltonian (Eq. H_h, Eq. ham-tj). Periodic extents must be >= 3. */
typedef struct {
  int32_t Lx, Ly;
  int32_t pbc_x, pbc_y;   /* 1 periodic, 0 open */
  int32_t n_up, n_dn;
  int32_t model;          /* SCALE_MODEL_* */
  double t, tp, U, J;     /* NN hopping, NNN hopping, on-site U (Hubbard), J (t-J) */
} scale_system;

/* Network shape and numerics. */
typedef struct {
  int32_t n_layers;       /* L >= 1 */
  int32_t h;              /* channels of every layer, 1..64 (ACE: of the conv blocks, 1..256;
                             wide SCALE: of the conv, 1..1024) */
  int32_t act;            /* SCALE_ACT_* */
  int32_t per_site_embed; /* 1: tables E_i per site (Sec. II.B); 0: one shared table */
  int32_t precision;      /* SCALE_PREC_FP64: everything FP64.
                             SCALE_PREC_MIXED: site-wise layers on the tensor cores as
                             three TF32 products of a hi/lo split (FP32 accumulation),
                             other layers, rank-r algebra and cached Phi^-1 in FP32,
                             LU / log|det| / drift check / E_loc sums in FP64.
                             SCALE_PREC_MIXED_FP16: as MIXED with three FP16 products
                             (m16n8k16: half the MMA instructions of TF32), the
                             activations scaled by 2^4 and each layer's weights by
                             the power of two that puts max|W| in [1/2, 1) so that the
                             lo parts stay normal, the accumulator scaled back exactly:
                             about 2^-21 per layer like MIXED; the site-wise
                             activations must stay below 4096 in magnitude. ACE and
                             wide shapes run it as MIXED.
                             SCALE_PREC_MIXED_BF16: as MIXED with three BF16 products
                             (about 2^-16 per layer instead of 2^-21).
                             The tensor-core path needs the SCALE layout and h in
                             {16, 32, 64}; otherwise the layers run in FP32 FMA.
                             ACE and wide shapes: when every layer has an mma.sync
                             fragment shape, MIXED runs the layers as the same three
                             TF32 products, on tcgen05 for the conv blocks of width 48,
                             144 or 192, the wide conv of width 384 or 640 (3x3 box or
                             5x5 plus) and the site-wise layers after them whose widths
                             are multiples of 128, on mma.sync for the rest; otherwise
                             every layer runs in FP32 FMA. Slater matrices and LU stay
                             FP64. */
  int32_t refresh_every;  /* FP64 re-factorisation of Phi every this many commits (>= 1);
                             counters start staggered at load (sample b at b mod
                             refresh_every) so refreshes spread evenly over calls */
  double drift_tol;       /* drift check threshold on the changed rows after a commit,
                             max_ab |M'_a . Binv'_b - delta_ab| / (|M'_a| |Binv'_b|)
                             (FP64, normalised backward error of the maintained
                             inverse); above it the sample is refreshed in FP64 within
                             the same call */
  int32_t ksize[SCALE_MAX_LAYERS];    /* odd kernel size per layer, 1 = site-wise */
  int32_t residual[SCALE_MAX_LAYERS]; /* 1: add the layer input (Eq. conv residual) */
  int32_t family;         /* SCALE_FAMILY_* (0 = SCALE) */
  int32_t n_conv;         /* ACE: layers [0, n_conv) are conv blocks (residual 1, odd ksize);
                             layers after them are site-wise (ksize 1, residual 0) */
  int32_t h_mlp;          /* ACE: width of the site-wise layers, 1..512 (wide SCALE 1..2048; 0 = h) */
  double ln_eps;          /* ACE: epsilon of the layer normalisation (>= 0) */
  int32_t stencil;        /* SCALE_STENCIL_*; the SCALE family's cached update takes layer 0 as a
                             1x1 or 3x3 box or the 5x5 plus (disk), other shapes run by full
                             recompute; scale_grad_logpsi takes either stencil */
  int32_t lowrank_kernel; /* kernel of the low-rank local energies: SCALE_LOWRANK_WARP (0, the
                             default) or SCALE_LOWRANK_BATCHED (1, mixed precision at 32
                             channels only; SCALE_EUNSUPPORTED otherwise) */
} scale_arch;

/* Low-rank local-energy kernels. WARP: one warp per connected configuration, the site-wise
 * layers of its affected sites on mma.sync tiles. BATCHED: the affected-site rows of all
 * moves of a walker packed into 128-row tiles and the site-wise layers run on tcgen05 (A
 * operand in Tensor Memory), move warps for the rest; the same results within the mixed-mode
 * tolerance. */
enum { SCALE_LOWRANK_WARP = 0, SCALE_LOWRANK_BATCHED = 1 };

typedef struct {
  int64_t n_eloc;          /* local energies produced (low-rank path) */
  int64_t n_eloc_full;     /* local energies produced (full-recompute path) */
  int64_t n_commits;       /* accepted moves applied */
  int64_t n_refresh;       /* samples re-factorised in FP64 */
  int64_t n_drift_refresh; /* of which forced by the drift check */
  double drift_max;        /* largest drift residual seen */
  int32_t batch;           /* samples currently loaded */
  int32_t max_moves;       /* capacity of connected configurations per sample */
  int32_t full_chunk;      /* configurations per chunk of the full-recompute path */
  int32_t wait_timeouts;   /* nonzero once a bounded wait of a tensor-core kernel ran out (its
                              outputs were NaN); cleared by reading */
} scale_stats;

typedef struct scale_ctx scale_ctx;

/* Number of float64 entries of the flat parameter vector for this shape. Returns -1 for
 * an invalid descriptor. Host-only, no GPU work. */
int64_t scale_param_count(const scale_system *sys, const scale_arch *arch);

/* Device bytes a context with this shape and batch capacity allocates (cache + scratch).
 * Host-only. Returns 0 for an invalid descriptor. */
size_t scale_footprint_bytes(const scale_system *sys, const scale_arch *arch, int32_t max_batch);

/* Create a context for up to max_batch samples on the current CUDA device.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream), used by every later call.
 * hbm_budget_bytes: 0 = no limit; otherwise SCALE_EBUDGET when the footprint exceeds it.
 * Validates the descriptors (SCALE_EINVAL) and allocates the cache (SCALE_ENOMEM). */
scale_status scale_create(const scale_system *sys, const scale_arch *arch, int32_t max_batch,
                          size_t hbm_budget_bytes, void *cuda_stream, scale_ctx **out);

/* Copy the parameters (params: scale_param_count float64 entries) and the reference
 * orbitals (M0: [2N][Ne] float64) into the context and build the derived tables
 * (precision copies, the layer-0 conv-of-embedding table). Invalidates loaded samples. */
scale_status scale_set_params(scale_ctx *ctx, const double *params, const double *M0);

/* Load B <= max_batch configurations occ[B][N] (int8) and build their cache: network
 * forward, Phi, FP64 Gauss-Jordan inverse with partial pivoting and log|det| (Sec. II.C,
 * "single LU"), projector P_s = W_s Phi^-1 and G0 = (M0 + proj_b) Phi^-1 (the part of every
 * Slater row's product with the inverse that does not depend on the network features).
 * sample_status[B] (int32, may be NULL)
 * receives SCALE_SAMPLE_* bits. */
scale_status scale_load(scale_ctx *ctx, const int8_t *occ, int32_t B, int32_t *sample_status);

/* log|psi| [B] (float64) and sign [B] (int32, 0 for a zero amplitude) of the loaded
 * samples, ascending-orbital convention. Either pointer may be NULL. */
scale_status scale_log_psi(scale_ctx *ctx, double *logabs, int32_t *sign);

/* Current configurations occ[B][N] (int8) of the loaded samples (changed by commits). */
scale_status scale_get_occ(scale_ctx *ctx, int8_t *occ);

/* Ratios psi(n')/psi(n) (ascending convention) for M moves per sample:
 * moves [B][M][4] int32, ratio [B][M] float64. Low-rank update (Eq. neighbor + Eq. SMW).
 * A move that leaves the model's space (occupied target, double occupancy in t-J) gives
 * ratio 0. Requires the SCALE layer layout (k_l = 1 for l >= 1), else SCALE_EUNSUPPORTED. */
scale_status scale_ratios(scale_ctx *ctx, const int32_t *moves, int32_t M, double *ratio);

/* E_loc [B] (float64) of the loaded samples.
 * path SCALE_PATH_LOWRANK: connected configurations enumerated on the device, each ratio a
 *   rank-r determinant against the cached Phi^-1 after an incremental receptive-field
 *   update of the network (needs k_l = 1 for l >= 1). At the wide shapes the affected rows
 *   of many moves are gathered and the site-wise layers run on them as row GEMMs (chunks of
 *   moves sized by the context's activation buffers); the call stays asynchronous.
 * path SCALE_PATH_FULL: psi(n) and every psi(n') by a full network forward in the mode's
 *   precision and a fresh FP64 LU with partial pivoting -- the comparison path of
 *   Sec. III.A, any layer layout; nothing cached by the context enters the result. The
 *   configurations run in chunks of max(max_batch, a memory-sized count of up to 4096), and
 *   the call stays asynchronous (the counts of connected configurations never reach the
 *   host). */
scale_status scale_local_energy(scale_ctx *ctx, int32_t path, double *eloc);

/* Apply one accepted move per sample (moves [B][4] int32, kind -1 = reject): Woodbury
 * update of Phi^-1 (Eq. SMW, second line), rank-r update of the projector and of G0, incremental
 * update of the cached features, occupations and slot maps, running log|det|. Samples
 * whose commit counter reaches refresh_every, or whose drift check fired, are
 * re-factorised in FP64 within the same call. Moves must be allowed (the library checks
 * and skips a move whose source is empty or whose target is occupied). */
scale_status scale_commit(scale_ctx *ctx, const int32_t *moves);

/* n_steps Metropolis steps of every loaded sample, drawing n from P(n) ~ |psi(n)|^2 by local
 * updates (Sec. II.A; the optimisation settings use 2.5 N steps per sample). Step k of
 * sample b proposes the hop of the pick[k][b]-th occupied orbital (ascending o = s*N + i,
 * pick in [0, Ne)) one site along dir[k][b] (0 +x, 1 -x, 2 +y, 3 -y); a target past an open
 * edge or already holding an electron of that spin (t-J: any electron) is rejected, else
 * the move is accepted when u[k][b] < |psi(n')/psi(n)|^2, the square of the rank-r
 * determinant against the cached inverse. An accepted move is committed as by
 * scale_commit (Woodbury update, drift check); a sample whose psi is zero accepts every
 * proposal and is re-factorised. Samples whose commit counter reaches refresh_every are
 * re-factorised in FP64 at the next multiple of 8 steps and at the end of the call (drift-
 * flagged ones after the step that flagged them). pick, dir: int32 [n_steps][B];
 * u: float64 [n_steps][B] in [0, 1), all random numbers supplied by the caller;
 * accepted: int32 [B], set to the number of accepted steps. Needs the SCALE layer layout
 * (SCALE_EUNSUPPORTED otherwise). */
scale_status scale_sweep(scale_ctx *ctx, int32_t n_steps, const int32_t *pick, const int32_t *dir,
                         const double *u, int32_t *accepted);

/* Symmetry-projected amplitude of the loaded samples (App. "Symmetry Projection"):
 *   psi_sym(n) = sum_g Pi(n, g) chi_g psi(g n).
 * perms: device int32 [G][2N] orbital permutations (o = s*N + i; g n occupies perms[g][o]
 * for each orbital o occupied in n; lattice symmetries move the site of both spins, spin
 * inversion exchanges s, and with n_up != n_dn its images leave the sector and give no
 * term). chi: device float64 [G] real characters (1 for the fully symmetric projection). Pi(n, g) is the parity of the permutation sorting the images
 * of n's occupied orbitals (ascending), the fermionic sign of the relabelling. Every psi(g n)
 * is a fresh network forward and FP64 LU (G evaluations per sample); the cached inverses and
 * features are left untouched. Outputs: logabs float64 [B] (log|psi_sym|, -inf when the sum
 * vanishes) and sign int32 [B]. An image outside the model's space (other particle numbers, a
 * t-J double occupancy, two occupied orbitals sent to one, or an occupied orbital sent outside
 * [0, 2N)) contributes 0. All pointers are device memory owned by the caller; the call is
 * asynchronous on the context's stream. SCALE_EINVAL: G < 1, a null pointer, or no parameters
 * or samples loaded. */
scale_status scale_log_psi_sym(scale_ctx *ctx, int32_t G, const int32_t *perms, const double *chi,
                               double *logabs, int32_t *sign);

/* Re-factorise in FP64 every loaded sample (force_all = 1) or only the ones flagged by
 * the drift check or the commit counter (force_all = 0). */
scale_status scale_refresh(scale_ctx *ctx, int32_t force_all);

/* Per-sample gradients d log|psi| / d theta, grad [B][P] float64 (flat parameter
 * layout): d log|det Phi| / d Phi = Phi^-T, back through the projection, every layer and
 * the embedding (hand-written backward). recompute = 1 keeps only every ceil(sqrt(L))-th
 * layer input and recomputes the rest (for deep stacks that exceed the scratch).
 * SCALE family only (either stencil); ACE and the wide shapes return SCALE_EUNSUPPORTED. */
scale_status scale_grad_logpsi(scale_ctx *ctx, double *grad, int32_t recompute);

/* Test hook for the failure path of the tensor-core kernels (not a construct of the paper):
 * what = 1 makes the next local-energy call of a context that runs the batched tensor-core
 * kernel (mixed precision, 32 channels) leave the first hand-off between its warp roles
 * unsignalled, so that the bounded wait on it runs out: the affected walkers' E_loc come back
 * NaN and scale_get_stats reports wait_timeouts; no fault, trap or hang. One-shot; what = 0
 * clears it. SCALE_EUNSUPPORTED for contexts that do not run that kernel. */
scale_status scale_test_inject(scale_ctx *ctx, int32_t what);

/* Counters since creation (host struct). Synchronises the context's stream. */
scale_status scale_get_stats(scale_ctx *ctx, scale_stats *out_host);

/* Text of the last error of this context ("" if none); valid until the next call. */
const char *scale_last_error(scale_ctx *ctx);

/* Free the context and its device memory (synchronises its stream). NULL is a no-op. */
void scale_destroy(scale_ctx *ctx);

/* log|psi| [B] and sign [B] (ascending convention, as scale_log_psi) of B configurations
 * occ[B][N] for the given shape, parameters and reference orbitals, WITHOUT any device
 * allocation by the call and without a context: for callers that cannot call cudaMalloc
 * (code running under a memory pool or arena owned by another runtime, plugins inside a
 * host application, code that may not allocate after setup). The paper has no counterpart;
 * this is a packaging of the load path (forward, Slater matrices, FP64 LU with partial
 * pivoting) for such callers.
 * All pointers are device pointers owned by the caller: params (scale_param_count
 * float64), M0 ([2N][Ne] float64), occ, logabs, sign. The working memory is one 64 MiB
 * file-scope device array of the library that every GPU loading it holds until the process
 * exits; larger batches are processed in chunks within the call, and a shape whose single
 * sample does not fit returns SCALE_EBUDGET. Every call shares that array and leaves its
 * contents behind: calls that overlap on the GPU (other streams or host threads on the same
 * device) race and must be serialised by the caller. The first call on a device looks up the
 * array's device address with that device current (cudaGetSymbolAddress) and caches it for
 * the device's current CUDA context; a call made under another context of the device (after
 * cudaDeviceReset, or a context the caller made current) looks it up again. Make the first
 * call on a device, and the first after such a change, before any stream capture. Work is
 * enqueued on cuda_stream (NULL = legacy stream). SCALE_EUNSUPPORTED for the ACE and wide
 * families. Per-sample problems as in scale_log_psi (-inf, sign 0). */
scale_status scale_log_psi_noalloc(const scale_system *sys, const scale_arch *arch, const double *params,
                                   const double *M0, const int8_t *occ, int32_t B, double *logabs,
                                   int32_t *sign, void *cuda_stream);

/* ------------------------------------------------------------------------------------
 * Serving: continuous batching of local-energy and amplitude requests from many Markov
 * chains, on lattices of different sizes and dopings, with device-resident chain state.
 * Not a construct of the paper (it has no serving layer); it drives the same kernels.
 *
 * A server owns one context per class (system + network + parameters) with a pool of
 * walker slots. SCALE_SRV_OPEN loads a chain's walkers into free slots; the walkers'
 * configuration, Phi^-1, projector and cached features stay in HBM until SCALE_SRV_CLOSE.
 * Requests (ELOC: local energies; STEP: local energies, then one Woodbury commit per
 * walker with the given moves; LOGPSI: log|psi|) that arrive while a class's batch is on
 * the GPU are merged into that class's next batch (one request per chain per batch);
 * classes run on their own CUDA streams and overlap on the device. A chain is admitted
 * when its class has enough free slots and the resident footprint of all open chains plus
 * its own stays within hbm_budget_bytes; until then it waits in arrival order. Results are
 * bit-identical to serving the chain alone: every walker is computed by its own CTA.
 * Scheduling runs on one host thread; no kernel waits on the host.
 * ------------------------------------------------------------------------------------ */
enum { SCALE_SRV_OPEN = 0, SCALE_SRV_ELOC = 1, SCALE_SRV_STEP = 2, SCALE_SRV_LOGPSI = 3, SCALE_SRV_CLOSE = 4 };

typedef struct scale_server scale_server;

typedef struct {
  int32_t n_classes;
  const scale_system *sys;     /* [n_classes] host array */
  const scale_arch *arch;      /* [n_classes] host array; SCALE layer layout required */
  const double *const *params; /* [n_classes] device pointers (copied at creation) */
  const double *const *M0;     /* [n_classes] device pointers (copied at creation) */
  const int32_t *slots;        /* [n_classes] walker slots per class (<= 65535) */
  size_t hbm_budget_bytes;     /* limit on the footprint of open chains, 0 = none */
} scale_server_cfg;

typedef struct {
  int32_t op;               /* SCALE_SRV_* */
  int32_t cls;              /* OPEN: class index */
  int32_t n_walkers;        /* OPEN: walkers of the chain */
  uint64_t chain;           /* ELOC / STEP / LOGPSI / CLOSE: the OPEN request's ticket */
  const int8_t *occ_host;   /* OPEN: [n_walkers][N], copied at submission */
  const int32_t *moves_host;/* STEP: [n_walkers][4], copied at submission */
  double *out_host;         /* ELOC / STEP: E_loc [n_walkers]; LOGPSI: log|psi| (-inf for a
                               zero amplitude); written before the ticket completes, must
                               stay valid until then */
} scale_request;

typedef struct {
  int32_t status;      /* SCALE_OK or the failure of this request */
  double latency_us;   /* submission to completion */
  uint64_t chain;      /* chain id (OPEN) */
} scale_result;

typedef struct {
  size_t resident_bytes, resident_max_bytes, budget_bytes;
  int64_t n_batches, n_requests, open_chains;
} scale_server_stats_t;

/* Create the server: one context and CUDA stream per class, all allocated up front, and
 * the scheduling thread. Errors as scale_create (SCALE_EUNSUPPORTED for a non-SCALE layer
 * layout). */
scale_status scale_server_create(const scale_server_cfg *cfg, scale_server **out);

/* Non-blocking submission; *ticket identifies the request (and, for OPEN, the chain).
 * SCALE_EBUDGET when an OPEN could never fit (more walkers than slots or than the budget),
 * SCALE_EINVAL for an unknown chain or malformed request. */
scale_status scale_server_submit(scale_server *srv, const scale_request *req, uint64_t *ticket);

/* Wait at most timeout_us for a ticket; SCALE_ETIMEOUT if it is still pending (the ticket
 * stays valid and its request keeps running). On completion fills *out and releases the
 * ticket. */
scale_status scale_server_poll(scale_server *srv, uint64_t ticket, scale_result *out, int32_t timeout_us);

/* Cancel a request that has not started: an ELOC / STEP / LOGPSI / CLOSE request still waiting
 * for its chain or its class's next batch, or an OPEN still waiting for admission. The ticket
 * completes at once with status SCALE_ECANCELED (poll it to release it; out_host is not
 * written, a cancelled STEP commits nothing); a cancelled OPEN makes the chain's later requests
 * fail with SCALE_EINVAL. SCALE_EINVAL when the ticket is unknown, already on the GPU or done
 * (such a request runs to completion). Never blocks on the GPU. */
scale_status scale_server_cancel(scale_server *srv, uint64_t ticket);

/* Resident footprint, its maximum so far, batches and requests processed. */
scale_status scale_server_stats(scale_server *srv, scale_server_stats_t *out);

/* Stop the scheduler, wait for the streams, free everything. NULL is a no-op. */
void scale_server_destroy(scale_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* SCALE_H */
