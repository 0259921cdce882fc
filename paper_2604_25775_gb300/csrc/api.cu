// api.cu -- the C ABI of include/scale.h: descriptor validation, context allocation
// (one cudaMalloc per buffer at creation), parameter upload and the call sequences.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "mlp_mma.cuh"
#include "scale_internal.cuh"

using namespace scale;

namespace {

#define SCALE_TRY(ctx, expr)                                                              \
  do {                                                                                    \
    cudaError_t _e = (expr);                                                              \
    if (_e != cudaSuccess) {                                                              \
      (ctx)->err = std::string("CUDA error in ") + #expr + ": " + cudaGetErrorString(_e); \
      return SCALE_ECUDA;                                                                 \
    }                                                                                     \
  } while (0)

bool validate(const scale_system* s, const scale_arch* a, std::string* why) {
  char buf[256];
  auto fail = [&](const char* m) {
    *why = m;
    return false;
  };
  if (!s || !a) return fail("null descriptor");
  if (s->Lx < 1 || s->Ly < 1 || s->Lx > 128 || s->Ly > 128) return fail("lattice extents must be in [1, 128]");
  if ((s->pbc_x && s->Lx < 3) || (s->pbc_y && s->Ly < 3)) return fail("periodic extents must be >= 3");
  const int N = s->Lx * s->Ly;
  if (N > 4096) return fail("at most 4096 sites");
  if (s->n_up < 0 || s->n_dn < 0 || s->n_up > N || s->n_dn > N || s->n_up + s->n_dn < 1)
    return fail("particle numbers out of range");
  if (s->model != SCALE_MODEL_HUBBARD && s->model != SCALE_MODEL_TJ && s->model != SCALE_MODEL_HUBBARD_PH)
    return fail("unknown model");
  if (s->model == SCALE_MODEL_HUBBARD_PH && s->tp != 0.0)
    return fail("particle-hole transformed model: t' must be 0 (the transformation keeps the hopping form "
                "on nearest-neighbour bonds only)");
  if (s->model == SCALE_MODEL_TJ && s->n_up + s->n_dn > N) return fail("t-J: more electrons than sites");
  if (a->n_layers < 1 || a->n_layers > SCALE_MAX_LAYERS) return fail("n_layers must be in [1, 32]");
  if (a->family != SCALE_FAMILY_SCALE && a->family != SCALE_FAMILY_ACE && a->family != SCALE_FAMILY_WIDE)
    return fail("unknown network family");
  if (a->stencil != SCALE_STENCIL_BOX && a->stencil != SCALE_STENCIL_DISK) return fail("unknown stencil");
  if (a->family == SCALE_FAMILY_ACE || a->family == SCALE_FAMILY_WIDE) {
    const bool ace = a->family == SCALE_FAMILY_ACE;
    if (a->h < 1 || a->h > (ace ? kAceMaxH : kWideMaxH))
      return fail(ace ? "ACE: h must be in [1, 256]" : "wide SCALE: h must be in [1, 1024]");
    if (a->n_conv < 1 || a->n_conv > a->n_layers) return fail("n_conv must be in [1, n_layers]");
    if (a->n_layers > a->n_conv && (a->h_mlp < 0 || a->h_mlp > (ace ? kAceMaxHMlp : kWideMaxHMlp)))
      return fail(ace ? "ACE: h_mlp must be in [0, 512]" : "wide SCALE: h_mlp must be in [0, 2048]");
    if (ace && !(a->ln_eps >= 0.0)) return fail("ACE: ln_eps must be >= 0");
    for (int l = 0; l < a->n_layers; ++l) {
      const bool conv = l < a->n_conv;
      if (ace && conv && a->residual[l] != 1) return fail("ACE: conv blocks carry the residual (Eq. ACE)");
      if (!conv && (a->ksize[l] != 1 || a->residual[l] != 0))
        return fail("layers after the conv blocks are site-wise (kernel size 1, no residual)");
    }
  } else {
    if (a->h < 1 || a->h > kMaxH) return fail("h must be in [1, 64]");
  }
  if (a->act != SCALE_ACT_TANH && a->act != SCALE_ACT_SILU) return fail("unknown activation");
  if (a->precision != SCALE_PREC_FP64 && a->precision != SCALE_PREC_MIXED && a->precision != SCALE_PREC_MIXED_BF16 &&
      a->precision != SCALE_PREC_MIXED_FP16)
    return fail("unknown precision");
  if (a->refresh_every < 1) return fail("refresh_every must be >= 1");
  if (a->lowrank_kernel != SCALE_LOWRANK_WARP && a->lowrank_kernel != SCALE_LOWRANK_BATCHED)
    return fail("unknown low-rank kernel");
  for (int l = 0; l < a->n_layers; ++l) {
    const int k = a->ksize[l];
    if (k < 1 || k > 7 || (k % 2) == 0) {
      snprintf(buf, sizeof buf, "layer %d: kernel size must be odd in [1, 7]", l);
      *why = buf;
      return false;
    }
    if (a->residual[l] != 0 && a->residual[l] != 1) return fail("residual flags must be 0 or 1");
  }
  return true;
}

int64_t param_count(const scale_system* s, const scale_arch* a) {
  const int64_t N = (int64_t)s->Lx * s->Ly, h = a->h, Ne = s->n_up + s->n_dn;
  int64_t n = (a->per_site_embed ? N : 1) * 4 * h;
  if (a->family != SCALE_FAMILY_SCALE) {
    const bool ln = a->family == SCALE_FAMILY_ACE;
    for (int l = 0; l < a->n_layers; ++l) {
      const int64_t ci = ace_width_in(*a, l), co = ace_width_out(*a, l);
      n += (int64_t)stencil_taps(a->stencil, a->ksize[l]) * ci * co + co + (ln && l < a->n_conv ? 2 * co : 0);
    }
    return n + (int64_t)ace_width_out(*a, a->n_layers - 1) * 2 * Ne + 2 * Ne;
  }
  for (int l = 0; l < a->n_layers; ++l) n += (int64_t)stencil_taps(a->stencil, a->ksize[l]) * h * h + h;
  return n + h * 2 * Ne + 2 * Ne;
}

// Bonds of Eq. H_h: NN (i, i+x), (i, i+y); NNN (i, i+x+y), (i, i+x-y); open edges dropped.
std::vector<int32_t> make_bonds(const Lattice& lat, int* nb_nn, int* nb_nnn) {
  std::vector<int32_t> out;
  const int offs[4][2] = {{1, 0}, {0, 1}, {1, 1}, {1, -1}};
  *nb_nn = *nb_nnn = 0;
  for (int kind = 0; kind < 2; ++kind) {
    if (kind == 1 && lat.tp == 0.0) break;
    for (int i = 0; i < lat.N; ++i)
      for (int d = 0; d < 2; ++d) {
        const int j = site_off(lat, i, offs[2 * kind + d][0], offs[2 * kind + d][1]);
        if (j < 0) continue;
        out.push_back(i);
        out.push_back(j);
        ++(kind == 0 ? *nb_nn : *nb_nnn);
      }
  }
  return out;
}

struct Sizes {
  size_t T, total;
  int cap;
  int full_chunk;  // configurations per full-recompute chunk
  size_t fc;       // entries of the chunk-sized scratch: max(max_batch, full_chunk)
};

// The full-recompute path evaluates its configurations in chunks whose scratch (FP64 Slater
// matrix, two activation buffers, packed occupations) stays within about 1 GiB, at most 4096
// configurations: enough determinant CTAs to fill every SM whatever the context's batch.
constexpr size_t kFullChunkBytes = size_t(1) << 30;
constexpr int kFullChunkMax = 4096;

Sizes sizes_of(const scale_system* s, const scale_arch* a, int B) {
  Sizes z{};
  const size_t N = (size_t)s->Lx * s->Ly, Ne = s->n_up + s->n_dn, h = a->h;
  z.T = a->precision == SCALE_PREC_FP64 ? 8 : 4;
  const size_t T = z.T;
  const size_t nb_nn = 2 * N, nb_nnn = s->tp != 0.0 ? 2 * N : 0;  // upper bounds
  z.cap = (int)(2 * (nb_nn + nb_nnn) + (s->model == SCALE_MODEL_TJ ? nb_nn : 0));
  const size_t P = (size_t)param_count(s, a);
  const size_t k0 = a->ksize[0];
  const bool ace = a->family != SCALE_FAMILY_SCALE;
  // ACE / wide activations: the widest layer, in mixed precision as (hi, lo) halves
  // (tensor-core layers keep their rows split between them)
  const size_t hmax = ace ? (T == 4 ? 2 : 1) * std::max<size_t>(h, (size_t)ace_width_out(*a, a->n_layers - 1)) : h;
  const size_t per_cfg = Ne * Ne * 8 + 2 * N * hmax * T + N + 4 * 4;
  z.full_chunk = (int)std::max<size_t>(1, std::min<size_t>(kFullChunkMax, kFullChunkBytes / per_cfg));
  z.fc = std::max<size_t>((size_t)B, (size_t)z.full_chunk);
  const size_t FC = z.fc;
  size_t t = 0;
  t += P * 8 + (T == 4 ? P * 4 : 0);
  t += 2 * N * Ne * 8 + (T == 4 ? 2 * N * Ne * 4 : 0) + 2 * N * Ne * T;
  // the cached update: narrow SCALE, or the wide shapes with a layer layout it covers
  const bool cached = !ace || wide_lowrank_shapes(*a);
  const size_t hl = ace ? (size_t)ace_width_out(*a, a->n_layers - 1) : h;  // width of H(L)
  t += cached ? (a->per_site_embed ? N : 1) * 4 * stencil_taps(a->stencil, (int)k0) * h * T : 16;  // KE
  t += (nb_nn + nb_nnn) * 2 * 4;
  t += (size_t)B * (N + Ne * 4 + 2 * N * 4);
  t += cached ? (size_t)B * N * (h + hl) * T : 32;  // z0, HL
  t += FC * N * hmax * T * 2;                       // act_a, act_b
  t += cached ? (size_t)B * Ne * Ne * T : 16;       // Binv
  t += cached ? (size_t)B * 2 * Ne * hl * T : 16;   // Pt
  if (ace && cached) t += (FC * N / (size_t)wide_rows_per_move(*s, *a) + 1) * wide_meta_bytes();  // move records
  t += (size_t)B * (8 + 4 + 4 + 4 + 8 + 4 + 4 + 8 + 4 + 8);
  t += FC * Ne * Ne * 8;                   // Phi64
  t += ace ? 16 : (size_t)B * commit_scratch_elems((int)Ne, (int)N) * T;  // commit scratch
  t += ace ? 16 : (size_t)B * Ne * 2 * N * T;                            // G0t
  if (ace && T == 4) t += ace_frag_bytes(*a);
  if (a->lowrank_kernel == SCALE_LOWRANK_BATCHED) t += (size_t)(a->n_layers - 1) * 2 * h * h * 4;  // weight image
  t += FC * (N + 4 + 8 + 4 + 4);          // full-path chunk: occupations, owner, log|psi|, sign, list
  t += (size_t)B * z.cap * (8 + 16);       // full-path coefficients, moves
  t += (size_t)B * (z.cap + 1) * (8 + 4);  // full-path log|psi| and sign of every entry
  t += (size_t)(B + 1) * 8 + 64;
  z.total = t;
  return z;
}

template <typename TD, typename TS>
__global__ void k_convert(const TS* __restrict__ in, TD* __restrict__ out, size_t n) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
    out[q] = (TD)in[q];
}

// M0b[o][k] = M0[o][k] + proj_b[s(o) * Ne + k]
template <typename T>
__global__ void k_m0b(const T* __restrict__ M0, const T* __restrict__ pb, int N, int Ne, T* __restrict__ out) {
  const size_t total = (size_t)2 * N * Ne;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const size_t o = q / Ne, k = q - o * Ne;
    out[q] = M0[q] + pb[(o / N) * Ne + k];
  }
}

template <typename P>
cudaError_t alloc(scale_ctx* c, P** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc((void**)ptr, bytes);
  if (e == cudaSuccess) c->allocated += bytes;
  return e;
}

void free_all(scale_ctx* c) {
  void* ptrs[] = {c->params64, c->params32, c->M0_64, c->M0_32, c->M0b, c->KE, c->bonds, c->occ, c->orb_of_slot,
                  c->slot_of_orb, c->z0, c->HL, c->Binv, c->Pt, c->logabs, c->sign_slot, c->status,
                  c->commits, c->drift, c->Phi64, c->act_a, c->act_b, c->list, c->list_count, c->stat_dev,
                  c->move_count, c->full_occ, c->full_owner, c->full_coeff, c->full_la_all, c->full_sg_all,
                  c->full_list, c->full_vcount, c->full_moves,
                  c->commit_scratch, c->la_tmp, c->sg_tmp, c->full_la, c->full_sg, c->full_diag,
                  c->full_offsets, c->grad_scratch, c->wfrag, c->ace_frag, c->ace_err, c->et_wimg, c->wl_meta, c->G0t};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

scale_status check_loaded(scale_ctx* c) {
  if (!c) return SCALE_EINVAL;
  if (!c->params_set) {
    c->err = "parameters not set (scale_set_params)";
    return SCALE_EINVAL;
  }
  if (c->B <= 0) {
    c->err = "no samples loaded (scale_load)";
    return SCALE_EINVAL;
  }
  return SCALE_OK;
}

scale_status require_lowrank(scale_ctx* c) {
  if (c->ace) {
    c->err = c->wide_lr ? "the wide SCALE shapes offer the cached local energies only (no ratios, commits, "
                          "sweeps or refreshes): use scale_local_energy"
                        : "this network family (ACE, or a wide layout without the SCALE layer pattern) has no "
                          "cached update: use the full-recompute path";
    return SCALE_EUNSUPPORTED;
  }
  if (!c->lowrank_ok) {
    c->err = "low-rank path needs the SCALE layer layout: layer 0 a 1x1 or 3x3 box or the 5x5 plus "
             "(disk stencil), site-wise layers (kernel size 1) after it; use the full-recompute path";
    return SCALE_EUNSUPPORTED;
  }
  return SCALE_OK;
}

}  // namespace

namespace scale {

// FP64 re-factorisation of the samples selected by the commit counter / drift flag (or
// all of them): network forward, ascending slot maps, Phi, Gauss-Jordan inverse, projector.
cudaError_t refresh_samples(scale_ctx* c, bool force_all, bool counters_due) {
  cudaError_t e;
  if ((e = launch_mark_refresh(c, force_all, counters_due)) != cudaSuccess) return e;
  if ((e = launch_forward(c, c->occ, c->B, c->list, true, c->Phi64, c->list_count)) != cudaSuccess) return e;
  if ((e = launch_slots_list(c, c->list, c->B)) != cudaSuccess) return e;
  if ((e = launch_gj(c, c->Phi64, c->Ne, c->B, c->list, true, c->fp64, c->Binv, c->logabs, c->sign_slot,
                     c->status)) != cudaSuccess)
    return e;
  return launch_projector(c, c->B, c->list, c->list_count);
}

}  // namespace scale

extern "C" {

int64_t scale_param_count(const scale_system* sys, const scale_arch* arch) {
  std::string why;
  if (!validate(sys, arch, &why)) return -1;
  return param_count(sys, arch);
}

size_t scale_footprint_bytes(const scale_system* sys, const scale_arch* arch, int32_t max_batch) {
  std::string why;
  if (!validate(sys, arch, &why) || max_batch < 1) return 0;
  return sizes_of(sys, arch, max_batch).total;
}

scale_status scale_create(const scale_system* sys, const scale_arch* arch, int32_t max_batch,
                          size_t hbm_budget_bytes, void* cuda_stream, scale_ctx** out) {
  if (!out) return SCALE_EINVAL;
  *out = nullptr;
  std::string why;
  if (!validate(sys, arch, &why) || max_batch < 1 || max_batch > 65535) return SCALE_EINVAL;
  const Sizes sz = sizes_of(sys, arch, max_batch);
  if (hbm_budget_bytes && sz.total > hbm_budget_bytes) return SCALE_EBUDGET;
  scale_ctx* c = new scale_ctx();
  c->sys = *sys;
  c->arch = *arch;
  c->N = sys->Lx * sys->Ly;
  c->Ne = sys->n_up + sys->n_dn;
  c->h = arch->h;
  c->L = arch->n_layers;
  c->k0 = arch->ksize[0];
  c->r0 = (c->k0 - 1) / 2;
  c->fp64 = arch->precision == SCALE_PREC_FP64;
  c->P = param_count(sys, arch);
  c->B_max = max_batch;
  c->stream = (cudaStream_t)cuda_stream;
  c->budget = hbm_budget_bytes;
  c->lat = Lattice{sys->Lx, sys->Ly, sys->pbc_x, sys->pbc_y, c->N, sys->n_up, sys->n_dn, c->Ne, sys->model,
                   sys->t, sys->tp, sys->U, sys->J};
  c->ace = arch->family != SCALE_FAMILY_SCALE;  // ACE and the wide SCALE shapes: full recompute
  // the cached update: layer 0 a 3x3 box or (disk stencil) up to the 13-site plus, so that the
  // pairs (touched site, tap) of a hop fit one warp and its affected sites kSMax
  c->lowrank_ok = !c->ace && (c->k0 <= 3 || (c->k0 == 5 && arch->stencil == SCALE_STENCIL_DISK));
  for (int l = 1; l < c->L; ++l) c->lowrank_ok = c->lowrank_ok && arch->ksize[l] == 1;
  c->hpad = c->h <= 16 ? 16 : (c->h <= 32 ? 32 : 64);
  c->use_mma = !c->fp64 && c->lowrank_ok && c->h == c->hpad;
  c->hmax = c->ace ? std::max(c->h, ace_width_out(*arch, c->L - 1)) : c->h;
  c->ace_mma = c->ace && !c->fp64 && ace_mma_shapes(*arch);
  c->ace_tc = c->ace_mma && ace_tc_shapes(*arch);
  c->wide_lr = c->ace && wide_lowrank_shapes(*arch);  // the cached local energies at the wide shapes
  std::vector<int32_t> bonds = make_bonds(c->lat, &c->nb_nn, &c->nb_nnn);
  c->max_moves = 2 * (c->nb_nn + c->nb_nnn) + (sys->model == SCALE_MODEL_TJ ? c->nb_nn : 0);
  c->full_chunk = (int)sz.fc;  // the chunk buffers hold FC configurations: use all of them
  const size_t B = max_batch, N = c->N, Ne = c->Ne, h = c->h, T = c->fp64 ? 8 : 4;
  const size_t FC = sz.fc;
  const size_t Ns = arch->per_site_embed ? N : 1;
  const size_t cap = std::max(1, c->max_moves);
  cudaError_t e = cudaSuccess;
  auto A = [&](auto** p, size_t bytes) {
    if (e == cudaSuccess) e = alloc(c, p, bytes);
  };
  A(&c->params64, c->P * 8);
  if (!c->fp64) A(&c->params32, c->P * 4);
  A(&c->M0_64, 2 * N * Ne * 8);
  if (!c->fp64) A(&c->M0_32, 2 * N * Ne * 4);
  A((char**)&c->M0b, 2 * N * Ne * T);
  const bool ace = c->ace;
  const bool cached = !ace || c->wide_lr;
  const size_t hmax = ace ? (c->fp64 ? 1 : 2) * (size_t)c->hmax : h;  // mixed: (hi, lo) halves
  const size_t hl = ace ? (size_t)ace_width_out(*arch, c->L - 1) : h;  // width of H(L)
  A((char**)&c->KE, cached ? Ns * 4 * stencil_taps(arch->stencil, c->k0) * h * T : 16);
  A(&c->bonds, std::max<size_t>(bonds.size(), 2) * 4);
  A(&c->occ, B * N);
  A(&c->orb_of_slot, B * Ne * 4);
  A(&c->slot_of_orb, B * 2 * N * 4);
  A((char**)&c->z0, cached ? B * N * h * T : 16);
  A((char**)&c->HL, cached ? B * N * hl * T : 16);
  A((char**)&c->Binv, cached ? B * Ne * Ne * T : 16);
  A((char**)&c->Pt, cached ? B * 2 * Ne * hl * T : 16);
  if (c->wide_lr) {  // moves per chunk: their row slots fill the activation buffers
    c->wl_rows = wide_rows_per_move(*sys, *arch);
    c->wl_chunk = (int)std::min<size_t>((FC * N) / (size_t)c->wl_rows, (size_t)1 << 20);
    A((char**)&c->wl_meta, ((size_t)c->wl_chunk + 1) * wide_meta_bytes());
  }
  A(&c->logabs, B * 8);
  A(&c->sign_slot, B * 4);
  A(&c->status, B * 4);
  A(&c->commits, B * 4);
  A(&c->drift, B * 8);
  A(&c->Phi64, FC * Ne * Ne * 8);
  A((char**)&c->act_a, FC * N * hmax * T);
  A((char**)&c->act_b, FC * N * hmax * T);
  A(&c->list, B * 4);
  A(&c->list_count, 16);
  A(&c->stat_dev, 4 * 8);
  A(&c->move_count, B * 4);
  A((char**)&c->commit_scratch, ace ? 16 : B * commit_scratch_elems((int)Ne, (int)N) * T);
  A((char**)&c->G0t, ace ? 16 : B * Ne * 2 * N * T);
  A(&c->la_tmp, B * 8);
  A(&c->sg_tmp, B * 4);
  A(&c->full_occ, FC * N);
  A(&c->full_owner, FC * 4);
  A(&c->full_list, FC * 4);
  A(&c->full_vcount, 16);
  A(&c->full_la, FC * 8);
  A(&c->full_sg, FC * 4);
  A(&c->full_diag, B * 8);
  A(&c->full_offsets, (B + 1) * 8);
  A(&c->full_coeff, B * cap * 8);
  A(&c->full_moves, B * cap * 16);
  A(&c->full_la_all, B * (cap + 1) * 8);
  A(&c->full_sg_all, B * (cap + 1) * 4);
  if (c->use_mma) A((char**)&c->wfrag, wfrag_bytes(c->L, c->hpad));
  if (c->ace_mma) A((char**)&c->ace_frag, ace_frag_bytes(*arch));
  A(&c->ace_err, 16);  // error word of the tensor-core kernels (bounded waits)
  {
    // the batched tensor-core local-energy kernel: its slot size and whether its plan fits
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int rows = c->lowrank_ok ? et_rows_per_move(c, bonds) : 0;
    if (arch->lowrank_kernel == SCALE_LOWRANK_BATCHED) {
      if (!et_supported(c, rows, optin)) {
        free_all(c);
        delete c;
        return SCALE_EUNSUPPORTED;
      }
      c->et_rows = rows;
      A((char**)&c->et_wimg, et_wimg_bytes(c));
    }
  }
  if (e != cudaSuccess) {
    free_all(c);
    delete c;
    return SCALE_ENOMEM;
  }
  if (!bonds.empty())
    e = cudaMemcpyAsync(c->bonds, bonds.data(), bonds.size() * 4, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->stat_dev, 0, 32, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->drift, 0, B * 8, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->commits, 0, B * 4, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->ace_err, 0, 16, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    free_all(c);
    delete c;
    return SCALE_ECUDA;
  }
  c->stats.max_moves = c->max_moves;
  c->stats.full_chunk = c->full_chunk;
  *out = c;
  return SCALE_OK;
}

scale_status scale_set_params(scale_ctx* c, const double* params, const double* M0) {
  if (!c || !params || !M0) return SCALE_EINVAL;
  const size_t N = c->N, Ne = c->Ne;
  SCALE_TRY(c, cudaMemcpyAsync(c->params64, params, c->P * 8, cudaMemcpyDeviceToDevice, c->stream));
  SCALE_TRY(c, cudaMemcpyAsync(c->M0_64, M0, 2 * N * Ne * 8, cudaMemcpyDeviceToDevice, c->stream));
  if (!c->fp64) {
    k_convert<float, double><<<1024, 256, 0, c->stream>>>(c->params64, c->params32, (size_t)c->P);
    k_convert<float, double><<<1024, 256, 0, c->stream>>>(c->M0_64, c->M0_32, 2 * N * Ne);
    SCALE_TRY(c, cudaGetLastError());
  }
  if (c->ace) {  // the tensor-core fragments; the wide shapes' layer-0 table and M0 + proj_b
    SCALE_TRY(c, launch_ace_build(c));
    if (c->wide_lr) SCALE_TRY(c, launch_wide_params(c));
    c->params_set = true;
    c->B = 0;
    return SCALE_OK;
  }
  SCALE_TRY(c, launch_build_ke(c));
  SCALE_TRY(c, launch_build_wfrag(c));
  SCALE_TRY(c, launch_build_et(c));
  if (c->fp64) {
    const Net<double> n = make_net<double>(c);
    k_m0b<double><<<512, 256, 0, c->stream>>>(n.M0, n.proj_b, c->N, c->Ne, (double*)c->M0b);
  } else {
    const Net<float> n = make_net<float>(c);
    k_m0b<float><<<512, 256, 0, c->stream>>>(n.M0, n.proj_b, c->N, c->Ne, (float*)c->M0b);
  }
  SCALE_TRY(c, cudaGetLastError());
  c->params_set = true;
  c->B = 0;
  return SCALE_OK;
}

scale_status scale_load(scale_ctx* c, const int8_t* occ, int32_t B, int32_t* sample_status) {
  if (!c || !occ || B < 1) return SCALE_EINVAL;
  if (!c->params_set) {
    c->err = "parameters not set (scale_set_params)";
    return SCALE_EINVAL;
  }
  if (B > c->B_max) {
    c->err = "batch larger than max_batch";
    return SCALE_EINVAL;
  }
  c->B = B;
  SCALE_TRY(c, cudaMemcpyAsync(c->occ, occ, (size_t)B * c->N, cudaMemcpyDeviceToDevice, c->stream));
  SCALE_TRY(c, cudaMemsetAsync(c->drift, 0, (size_t)B * 8, c->stream));
  SCALE_TRY(c, launch_slots(c, c->occ, B));
  SCALE_TRY(c, launch_forward(c, c->occ, B, nullptr, true, c->Phi64));
  if (c->wide_lr) {  // the wide cache: FP64 inverse, z0 from the layer-0 table, Pt = W Phi^-1
    SCALE_TRY(c, launch_gj(c, c->Phi64, c->Ne, B, nullptr, true, c->fp64, c->Binv, c->logabs, c->sign_slot, c->status));
    SCALE_TRY(c, launch_wide_cache(c, B));
  } else if (c->ace) {  // log|det| and sign only (FP64 LU); nothing is cached for updates
    SCALE_TRY(c, launch_gj(c, c->Phi64, c->Ne, B, nullptr, false, true, nullptr, c->logabs, c->sign_slot, c->status));
  } else {
    SCALE_TRY(c, launch_gj(c, c->Phi64, c->Ne, B, nullptr, true, c->fp64, c->Binv, c->logabs, c->sign_slot, c->status));
    SCALE_TRY(c, launch_projector(c, B, nullptr));
  }
  if (sample_status)
    SCALE_TRY(c, cudaMemcpyAsync(sample_status, c->status, (size_t)B * 4, cudaMemcpyDeviceToDevice, c->stream));
  c->stats.batch = B;
  return SCALE_OK;
}

scale_status scale_log_psi(scale_ctx* c, double* logabs, int32_t* sign) {
  scale_status s = check_loaded(c);
  if (s != SCALE_OK) return s;
  SCALE_TRY(c, launch_logpsi_out(c, logabs, sign));
  return SCALE_OK;
}

scale_status scale_get_occ(scale_ctx* c, int8_t* occ) {
  scale_status s = check_loaded(c);
  if (s != SCALE_OK) return s;
  if (!occ) return SCALE_EINVAL;
  SCALE_TRY(c, cudaMemcpyAsync(occ, c->occ, (size_t)c->B * c->N, cudaMemcpyDeviceToDevice, c->stream));
  return SCALE_OK;
}

scale_status scale_ratios(scale_ctx* c, const int32_t* moves, int32_t M, double* ratio) {
  scale_status s = check_loaded(c);
  if (s != SCALE_OK) return s;
  if (!moves || !ratio || M < 1) return SCALE_EINVAL;
  if ((s = require_lowrank(c)) != SCALE_OK) return s;
  SCALE_TRY(c, launch_ratios(c, moves, M, ratio));
  return SCALE_OK;
}

scale_status scale_local_energy(scale_ctx* c, int32_t path, double* eloc) {
  scale_status s = check_loaded(c);
  if (s != SCALE_OK) return s;
  if (!eloc) return SCALE_EINVAL;
  if (path == SCALE_PATH_LOWRANK) {
    if (c->wide_lr) {
      SCALE_TRY(c, launch_wide_eloc(c, eloc));
    } else {
      if ((s = require_lowrank(c)) != SCALE_OK) return s;
      SCALE_TRY(c, launch_eloc_lowrank(c, eloc));
    }
    c->stats.n_eloc += c->B;
  } else if (path == SCALE_PATH_FULL) {
    SCALE_TRY(c, launch_eloc_full(c, eloc));
    c->stats.n_eloc_full += c->B;
  } else {
    return SCALE_EINVAL;
  }
  return SCALE_OK;
}

scale_status scale_commit(scale_ctx* c, const int32_t* moves) {
  scale_status s = check_loaded(c);
  if (s != SCALE_OK) return s;
  if (!moves) return SCALE_EINVAL;
  if ((s = require_lowrank(c)) != SCALE_OK) return s;
  SCALE_TRY(c, launch_commit(c, moves));
  SCALE_TRY(c, refresh_samples(c, false));
  return SCALE_OK;
}

scale_status scale_sweep(scale_ctx* c, int32_t n_steps, const int32_t* pick, const int32_t* dir, const double* u,
                         int32_t* accepted) {
  scale_status s = check_loaded(c);
  if (s != SCALE_OK) return s;
  if (n_steps < 0 || (n_steps > 0 && (!pick || !dir || !u)) || !accepted) return SCALE_EINVAL;
  if ((s = require_lowrank(c)) != SCALE_OK) return s;
  SCALE_TRY(c, cudaMemsetAsync(accepted, 0, sizeof(int32_t) * (size_t)c->B, c->stream));
  // Samples whose drift check fired, or whose step fell back to the occupations alone, are
  // re-factorised after the step that flagged them. Samples whose commit counter came due
  // wait for the next multiple of kSweepRefreshStride steps (and the end of the call), so
  // the FP64 refreshes of a sweep run as a few full launches instead of one thin launch
  // per step: one 224 x 224 FP64 inverse occupies an SM for milliseconds.
  constexpr int32_t kSweepRefreshStride = 8;
  for (int32_t k = 0; k < n_steps; ++k) {
    const size_t off = (size_t)k * c->B;
    SCALE_TRY(c, launch_metropolis(c, pick + off, dir + off, u + off, accepted));
    const bool due = (k % kSweepRefreshStride) == kSweepRefreshStride - 1 || k == n_steps - 1;
    SCALE_TRY(c, refresh_samples(c, false, due));
  }
  // The Metropolis commits leave the cached G0t rows behind the inverse (keeping them current
  // per accepted move costs more than the sweep's ratios save); one GEMM per sample restores them.
  if (n_steps > 0) SCALE_TRY(c, launch_build_g0(c, c->B, nullptr, nullptr));
  return SCALE_OK;
}

scale_status scale_log_psi_sym(scale_ctx* c, int32_t G, const int32_t* perms, const double* chi, double* logabs,
                               int32_t* sign) {
  scale_status s = check_loaded(c);
  if (s != SCALE_OK) return s;
  if (G < 1 || !perms || !chi || !logabs || !sign) return SCALE_EINVAL;
  SCALE_TRY(c, launch_log_psi_sym(c, G, perms, chi, logabs, sign));
  return SCALE_OK;
}

scale_status scale_refresh(scale_ctx* c, int32_t force_all) {
  scale_status s = check_loaded(c);
  if (s != SCALE_OK) return s;
  if ((s = require_lowrank(c)) != SCALE_OK) return s;
  SCALE_TRY(c, refresh_samples(c, force_all != 0));
  return SCALE_OK;
}

scale_status scale_grad_logpsi(scale_ctx* c, double* grad, int32_t recompute) {
  scale_status s = check_loaded(c);
  if (s != SCALE_OK) return s;
  if (!grad) return SCALE_EINVAL;
  if (c->ace) {
    c->err = "the per-sample gradient covers the SCALE family";
    return SCALE_EUNSUPPORTED;
  }
  SCALE_TRY(c, launch_grad(c, grad, recompute));
  return SCALE_OK;
}

scale_status scale_test_inject(scale_ctx* c, int32_t what) {
  if (!c || what < 0 || what > 1) return SCALE_EINVAL;
  if (!c->et_wimg) {
    c->err = "the batched tensor-core local-energy kernel does not run for this context";
    return SCALE_EUNSUPPORTED;
  }
  c->et_inject = what;
  return SCALE_OK;
}

scale_status scale_get_stats(scale_ctx* c, scale_stats* out) {
  if (!c || !out) return SCALE_EINVAL;
  double host[4];
  int32_t timeouts = 0;
  SCALE_TRY(c, cudaMemcpyAsync(host, c->stat_dev, sizeof host, cudaMemcpyDeviceToHost, c->stream));
  SCALE_TRY(c, cudaMemcpyAsync(&timeouts, c->ace_err, sizeof timeouts, cudaMemcpyDeviceToHost, c->stream));
  SCALE_TRY(c, cudaMemsetAsync(c->ace_err, 0, sizeof timeouts, c->stream));
  SCALE_TRY(c, cudaStreamSynchronize(c->stream));
  *out = c->stats;
  out->drift_max = host[0];
  int32_t cnt[6];
  std::memcpy(cnt, &host[1], sizeof cnt);
  out->n_commits = cnt[0];
  out->n_refresh = cnt[1];
  out->n_drift_refresh = cnt[2];
  out->wait_timeouts = timeouts;
  return SCALE_OK;
}

const char* scale_last_error(scale_ctx* c) { return c ? c->err.c_str() : "null context"; }

void scale_destroy(scale_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
}

}  // extern "C"
