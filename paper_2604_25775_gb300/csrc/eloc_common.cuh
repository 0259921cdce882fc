// eloc_common.cuh -- pieces shared by the local-energy kernels of the cached update
// (Sec. II.C): the argument block, the connected-configuration enumeration order and the
// packed move format.
//
// Connected configurations are enumerated on the device in a fixed order (NN bonds, then NNN
// bonds, each with spin up then down; then t-J exchanges on NN bonds), and compacted chunk by
// chunk in that order. Per-move contributions are summed in enumeration order, so E_loc does
// not depend on which warp evaluated which move.
#pragma once

#include "move.cuh"

namespace scale {

struct MoveDesc {
  int kind, src, dst, spin;
};

struct LowrankArgs {
  Lattice lat;
  int k0;
  const int8_t* occ;
  const int32_t* slot_of_orb;
  const void* z0;
  const void* HL;
  const void* Binv;
  const void* Pt;
  const void* G0t;
  const int32_t* bonds;
  int nb_nn, nb_nnn;
  const int32_t* status;
  double* out;           // eloc [B] or ratio [B][M]
  int32_t* move_count;   // [B] (eloc only)
  const int32_t* moves;  // explicit moves [B][M][4] (ratios only)
  int M;
  MlpFrags mf;
  const int32_t* list;   // optional: CTA i handles sample list[i]
};

// Candidate id -> move (kind -1 when not allowed in the current configuration) and its
// coefficient class: 0 NN hop (-t), 1 NNN hop (-t'), 2 exchange (-J/2).
__device__ __forceinline__ MoveDesc candidate(const LowrankArgs& a, const int8_t* occ, int id, int* cls) {
  MoveDesc m{-1, 0, 0, 0};
  const int nb = a.nb_nn + a.nb_nnn;
  if (id < 2 * nb) {
    const int q = id >> 1, s = id & 1;
    const int i = a.bonds[2 * q], j = a.bonds[2 * q + 1];
    const int oi = occ[i], oj = occ[j];
    const bool hi = (oi >> s) & 1, hj = (oj >> s) & 1;
    if (hi == hj) return m;
    const int src = hi ? i : j, dst = hi ? j : i;
    if (a.lat.model == SCALE_MODEL_TJ && occ[dst] != 0) return m;
    m.kind = 0;
    m.src = src;
    m.dst = dst;
    m.spin = s;
    *cls = (q < a.nb_nn) ? 0 : 1;
    return m;
  }
  const int q = id - 2 * nb;
  const int i = a.bonds[2 * q], j = a.bonds[2 * q + 1];
  const int oi = occ[i], oj = occ[j];
  if ((oi == 1 && oj == 2) || (oi == 2 && oj == 1)) {
    m.kind = 1;
    m.src = i;
    m.dst = j;
    m.spin = 0;
    *cls = 2;
  }
  return m;
}

// Moves of one chunk are kept packed in shared memory: bits 0-11 src, 12-23 dst (N <= 4096),
// 24 spin, 25 kind, 26-27 coefficient class.
constexpr int kMoveChunk = 1024;
__device__ __forceinline__ uint32_t pack_move(const MoveDesc& m, int cls) {
  return (uint32_t)m.src | ((uint32_t)m.dst << 12) | ((uint32_t)m.spin << 24) | ((uint32_t)m.kind << 25) |
         ((uint32_t)cls << 26);
}


__device__ __forceinline__ MoveDesc unpack_move(uint32_t pm) {
  MoveDesc m;
  m.src = (int)(pm & 0xfffu);
  m.dst = (int)((pm >> 12) & 0xfffu);
  m.spin = (int)((pm >> 24) & 1u);
  m.kind = (int)((pm >> 25) & 1u);
  return m;
}

// Coefficient of a packed move in slot order (the hop's Jordan-Wigner sign cancels against the
// row-permutation sign; the exchange element is -J/2 times det R).
__device__ __forceinline__ double move_coeff(const Lattice& lat, uint32_t pm) {
  const uint32_t cls = (pm >> 26) & 3u;
  return cls == 0 ? -lat.t : (cls == 1 ? -lat.tp : -0.5 * lat.J);
}

// Diagonal matrix element of configuration occ (shared-memory copy): Hubbard U * (doubly
// occupied sites); particle-hole Hubbard U * (sites with an up particle and no transformed
// down particle); t-J J sum_<ij> Sz_i Sz_j over the NN bonds, as (J/4) sum s_i s_j with the
// integer s = n_up - n_dn. One thread: integer counts, one FP64 multiply (FP64 instructions
// are scarce on this GPU: the same loop over the bonds in FP64 kept the CTA waiting for about
// 0.2M cycles; a warp-wide version took the kernel's registers from 80 to 96).
__device__ __forceinline__ double diag_energy(const LowrankArgs& a, const int8_t* occ_s) {
  const int N = a.lat.N;
  int cnt = 0;
  if (a.lat.model == SCALE_MODEL_HUBBARD) {
    for (int i = 0; i < N; ++i) cnt += occ_s[i] == 3;
  } else if (a.lat.model == SCALE_MODEL_HUBBARD_PH) {
    for (int i = 0; i < N; ++i) cnt += occ_s[i] == 1;
  } else {
    for (int q = 0; q < a.nb_nn; ++q) {
      const int oi = occ_s[a.bonds[2 * q]], oj = occ_s[a.bonds[2 * q + 1]];
      cnt += ((oi & 1) - ((oi >> 1) & 1)) * ((oj & 1) - ((oj >> 1) & 1));
    }
  }
  return a.lat.model == SCALE_MODEL_TJ ? (0.25 * a.lat.J) * cnt : a.lat.U * cnt;
}

// Number of candidate ids of a sample: 2 (NN + NNN bonds) hops, then NN exchanges (t-J).
__device__ __forceinline__ int candidate_count(const LowrankArgs& a) {
  const int nb = a.nb_nn + a.nb_nnn;
  return 2 * nb + ((a.lat.model == SCALE_MODEL_TJ && a.lat.J != 0.0) ? a.nb_nn : 0);
}

// Allowed moves among candidate ids [cs, ce), compacted into mlist in enumeration order by
// all NWARPS warps of the CTA; returns their number (every thread). warp_cnt: [NWARPS].
template <int NWARPS>
__device__ int enumerate_chunk(const LowrankArgs& a, const int8_t* occ_s, int cs, int ce, uint32_t* mlist,
                               int* warp_cnt) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int nm = 0;
  for (int sub = cs; sub < ce; sub += NWARPS * 32) {
    const int id = sub + tid;
    int cls = 0;
    MoveDesc m{-1, 0, 0, 0};
    if (id < ce) m = candidate(a, occ_s, id, &cls);
    const bool valid = m.kind >= 0;
    const unsigned bal = __ballot_sync(0xffffffffu, valid);
    if (lane == 0) warp_cnt[warp] = __popc(bal);
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < NWARPS; ++w) {
      if (w < warp) off += warp_cnt[w];
      tot += warp_cnt[w];
    }
    if (valid) mlist[nm + off + __popc(bal & ((1u << lane) - 1u))] = pack_move(m, cls);
    nm += tot;
    __syncthreads();
  }
  return nm;
}

inline LowrankArgs make_args(scale_ctx* c) {
  LowrankArgs a{};
  a.lat = c->lat;
  a.k0 = c->k0;
  a.occ = c->occ;
  a.slot_of_orb = c->slot_of_orb;
  a.z0 = c->z0;
  a.HL = c->HL;
  a.Binv = c->Binv;
  a.Pt = c->Pt;
  a.G0t = c->G0t;
  a.bonds = c->bonds;
  a.nb_nn = c->nb_nn;
  a.nb_nnn = c->nb_nnn;
  a.status = c->status;
  a.mf.wf = c->use_mma ? (const WFrag*)c->wfrag : nullptr;
  a.mf.kind = mma_kind_of(c->arch.precision);
  a.mf.oscale = c->use_mma && a.mf.kind == kFP16 ? fp16_scales(c) + kMaxLayers : nullptr;
  return a;
}

}  // namespace scale
