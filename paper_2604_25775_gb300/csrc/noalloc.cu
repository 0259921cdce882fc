// noalloc.cu -- log|psi| for a batch without any device allocation by the call.
//
// For callers that cannot call cudaMalloc: code running under a memory pool or arena that
// another runtime owns (an embedding framework, a plugin inside a host application), code
// that must not allocate between setup and teardown, or a caller with a fixed device
// budget that it reserved up front. They pass inputs and outputs only; the working memory
// of the evaluation (per-sample activations, the FP64 Slater matrices and the Gauss-Jordan
// work rows, slot maps, the precision copies of the parameters) lives in one file-scope
// device array of kNoAllocBytes (64 MiB) that every GPU loading this library holds until the
// process exits. A batch larger than one chunk of that array is processed chunk by chunk in
// the same call; a shape whose single sample (plus the parameter copies) does not fit is
// rejected with SCALE_EBUDGET.
//
// The array is shared by every call: calls that overlap on the GPU (different streams, or
// different host threads on one device) race on it and must be serialised by the caller.
// Nothing in it needs to start at zero: every word a call reads was written earlier in the
// same call.
//
// The device address of the array is looked up once per CUDA context: on the first call made
// with a device current, and again on the first call after that device's context changed
// (cudaDeviceReset, or a caller that made another context of the device current). The cache
// is keyed on the context's process-unique ID, so an address from a destroyed context is never
// reused. Make that first call on a device (and the first after a reset) outside any stream
// capture.
#include <cuda.h>

#include <cstring>
#include <mutex>

#include "mlp_mma.cuh"
#include "scale_internal.cuh"

using namespace scale;

namespace {

constexpr size_t kNoAllocBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct ScratchAddr {
  unsigned long long ctx_id;  // ID of the context the address belongs to
  void* ptr;
};
ScratchAddr g_scratch[kMaxDevices] = {};

// ID of the current CUDA context (driver entry points fetched through the runtime, so the
// library needs no link against the driver library). false when there is none yet or the
// driver lacks the calls.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
bool current_ctx_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool tried = false;
  if (!tried) {  // under g_mu
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (CtxGetCurrentFn)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (CtxGetIdFn)f;
  }
  if (!get_current || !get_id) return false;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

template <typename TD, typename TS>
__global__ void k_convert_na(const TS* __restrict__ in, TD* __restrict__ out, size_t n) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
    out[q] = (TD)in[q];
}

}  // namespace

extern "C" scale_status scale_log_psi_noalloc(const scale_system* sys, const scale_arch* arch, const double* params,
                                              const double* M0, const int8_t* occ, int32_t B, double* logabs,
                                              int32_t* sign, void* cuda_stream) {
  if (!sys || !arch || !params || !M0 || !occ || !logabs || !sign || B < 1) return SCALE_EINVAL;
  const int64_t P = scale_param_count(sys, arch);
  if (P < 0) return SCALE_EINVAL;
  if (arch->family != SCALE_FAMILY_SCALE) return SCALE_EUNSUPPORTED;  // no ACE working set here
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SCALE_ECUDA;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    unsigned long long id = 0;
    bool known = current_ctx_id(&id);
    if (!known || !g_scratch[dev].ptr || g_scratch[dev].ctx_id != id) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SCALE_ECUDA;
      if (!known) known = current_ctx_id(&id);  // the lookup made the device's context current
      // without a context ID the address is looked up again on every call
      g_scratch[dev] = known ? ScratchAddr{id, p} : ScratchAddr{0, nullptr};
      base = (unsigned char*)p;
    } else {
      base = (unsigned char*)g_scratch[dev].ptr;
    }
  }
  // a host-side context whose device pointers all point into the static array or at the
  // caller's buffers
  scale_ctx c;
  c.sys = *sys;
  c.arch = *arch;
  c.N = sys->Lx * sys->Ly;
  c.Ne = sys->n_up + sys->n_dn;
  c.h = arch->h;
  c.L = arch->n_layers;
  c.k0 = arch->ksize[0];
  c.fp64 = arch->precision == SCALE_PREC_FP64;
  c.P = P;
  c.stream = (cudaStream_t)cuda_stream;
  c.lat = Lattice{sys->Lx, sys->Ly, sys->pbc_x, sys->pbc_y, c.N, sys->n_up, sys->n_dn, c.Ne, sys->model,
                  sys->t, sys->tp, sys->U, sys->J};
  c.lowrank_ok = c.k0 <= 3 || (c.k0 == 5 && arch->stencil == SCALE_STENCIL_DISK);
  for (int l = 1; l < c.L; ++l) c.lowrank_ok = c.lowrank_ok && arch->ksize[l] == 1;
  c.hpad = c.h <= 16 ? 16 : (c.h <= 32 ? 32 : 64);
  c.use_mma = !c.fp64 && c.lowrank_ok && c.h == c.hpad;
  const size_t N = c.N, Ne = c.Ne, h = c.h, T = c.fp64 ? 8 : 4;
  // fixed part: parameter / reference-orbital copies and mma fragments
  size_t off = 0;
  c.params64 = const_cast<double*>(params);
  c.M0_64 = const_cast<double*>(M0);
  if (!c.fp64) {
    c.params32 = (float*)(base + off);
    off = align256(off + (size_t)P * 4);
    c.M0_32 = (float*)(base + off);
    off = align256(off + 2 * N * Ne * 4);
  }
  if (c.use_mma) {
    c.wfrag = base + off;
    off = align256(off + wfrag_bytes(c.L, c.hpad));
  }
  // per-sample part
  const size_t per = align256(N * h * T) * 2 + align256(Ne * Ne * 8) + align256(Ne * 4) + align256(2 * N * 4) +
                     align256(8) + 3 * align256(4);
  // nine per-sample buffers, each rounded up to 256 bytes once per chunk
  if (off + per + 9 * 256 > kNoAllocBytes) return SCALE_EBUDGET;
  const int chunk = (int)std::min<size_t>((kNoAllocBytes - off - 9 * 256) / per, 65535);
  if (chunk < 1) return SCALE_EBUDGET;
  if (!c.fp64) {
    k_convert_na<float, double><<<256, 256, 0, c.stream>>>(params, c.params32, (size_t)P);
    k_convert_na<float, double><<<256, 256, 0, c.stream>>>(M0, c.M0_32, 2 * N * Ne);
    if (cudaGetLastError() != cudaSuccess) return SCALE_ECUDA;
  }
  if (launch_build_wfrag(&c) != cudaSuccess) return SCALE_ECUDA;
  const int nb = chunk;
  auto take = [&](size_t bytes) {
    void* p = base + off;
    off = align256(off + bytes);
    return p;
  };
  c.act_a = take((size_t)nb * N * h * T);
  c.act_b = take((size_t)nb * N * h * T);
  c.Phi64 = (double*)take((size_t)nb * Ne * Ne * 8);
  c.orb_of_slot = (int32_t*)take((size_t)nb * Ne * 4);
  c.slot_of_orb = (int32_t*)take((size_t)nb * 2 * N * 4);
  c.logabs = (double*)take((size_t)nb * 8);
  c.sign_slot = (int32_t*)take((size_t)nb * 4);
  c.status = (int32_t*)take((size_t)nb * 4);
  c.commits = (int32_t*)take((size_t)nb * 4);
  if (off > kNoAllocBytes) return SCALE_EBUDGET;
  for (int b0 = 0; b0 < B; b0 += chunk) {
    const int n = std::min(chunk, B - b0);
    const int8_t* o = occ + (size_t)b0 * N;
    c.B = n;
    if (launch_slots(&c, o, n) != cudaSuccess) return SCALE_ECUDA;
    if (launch_forward(&c, o, n, nullptr, false, c.Phi64) != cudaSuccess) return SCALE_ECUDA;
    if (launch_gj(&c, c.Phi64, c.Ne, n, nullptr, false, true, nullptr, c.logabs, c.sign_slot, c.status) !=
        cudaSuccess)
      return SCALE_ECUDA;
    if (launch_logpsi_out(&c, logabs + b0, sign + b0) != cudaSuccess) return SCALE_ECUDA;
  }
  // the host-side context owns nothing
  c.params64 = nullptr;
  c.M0_64 = nullptr;
  return SCALE_OK;
}
