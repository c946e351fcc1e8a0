// Fused mixed-precision (complex64) Hamiltonian path: pruned z-column FFTs, one plane
// kernel per z-plane holding the (x, y) plane in shared memory with the potential and
// the projector add fused between the inverse and forward transforms, and the kinetic
// term fused into the last transform.
#pragma once

#include <memory>
#include <vector>

#include "engine.h"
#include "kernels.h"

namespace ks {

// Taylor accumulation fused into the last kernel of an H application (Eq. 8, the shared powers
// of the real-time step): as each value h of H psi is formed, acc1 <- base + a1 h and, when acc2
// is set, acc2 <- base + a2 h, with base the given block, or each accumulator's own old value when
// base is null.  base_is_psi: base is the H application's own input (its values are already in
// registers).  skip_h: H psi itself is not stored (the last power of a Taylor series).
// Power-sum form (nsum = 4, the fourth power of a Taylor-4 series whose earlier powers were
// kept): acc1 <- base + c1[0] w1 + c1[1] w2 + c1[2] psi + c1[3] h, with psi the H application's
// input (the third power, in registers), and acc2 likewise with c2 when set; the terms are added
// in this order, the same FP32 operations as four incremental updates of a stored accumulator.
struct TaylorEpi {
  float2* acc1 = nullptr;
  float2 a1{0.f, 0.f};
  float2* acc2 = nullptr;
  float2 a2{0.f, 0.f};
  const float2* base = nullptr;
  int base_is_psi = 0;
  int skip_h = 0;
  int nsum = 0;
  const float2* w1 = nullptr;
  const float2* w2 = nullptr;
  float2 c1[4] = {};
  float2 c2[4] = {};
};

class FusedOps {
 public:
  virtual ~FusedOps() = default;
  // hpsi = H psi for n states with potential v (grid order); te (may be null): the Taylor
  // accumulators updated by the same pass.
  virtual void apply_h(const float2* psi, float2* hpsi, int n, const float* v, cudaStream_t s,
                       const TaylorEpi* te = nullptr) = 0;
  // nout = sum_k occ[k] |psi_k(r)|^2 (grid order).
  virtual void density(const float2* psi, int n, const double* occ, float* nout, cudaStream_t s) = 0;
  // out[b][z][x][y] = Omega^{1/2} psi_b(r) on the grid (plane-major: z slowest), the unscaled
  // inverse transform of n packed states, by the pruned z-columns and the in-SMEM y, x passes.
  virtual void real_space(const float2* psi, int n, float2* out, cudaStream_t s) = 0;
  // The atoms moved.  prepare_atoms forms the per-plane projector lists on the host from the
  // geometry's new sphere lists (no device work, so it may overlap kernels in flight);
  // set_atoms uploads them and rebuilds the projector block (t: the engine's re-uploaded
  // tables); the caller synchronises the streams that may still read the old lists first.
  // Synchronous.
  virtual void prepare_atoms() = 0;
  virtual void set_atoms(const DevTables<float>& t) = 0;
};

// One member of a packed H application: a block of states of one cell, its output and its
// potential (grid order), with the Taylor accumulators of the same pass.
struct FusedGroupItem {
  FusedOps* ops = nullptr;
  const float2* psi = nullptr;
  float2* hpsi = nullptr;
  int n = 0;
  const float* v = nullptr;
  TaylorEpi te{};
  // the cell's first column buffer already holds the z transform of these n states (a density
  // of the same block was the cell's last use of it): the z-transform launch is skipped when
  // every member of a launch has it
  bool cols_ready = false;
};

// H psi of several cells' blocks that share one grid geometry (same L, N and cutoff, so the same
// sphere, columns and twiddles), e.g. the real-time requests of a server on one grid: each
// cell's projections and potential layout, then one launch of each of the z, plane and z kernels
// over all members' states (up to eight members per launch).  Grids without the team plane
// kernel run the members one at a time.  Asynchronous on s.
void fused_apply_h_group(const std::vector<FusedGroupItem>& items, cudaStream_t s);
// True when two fused paths may share a packed launch.
bool fused_same_geometry(const FusedOps* a, const FusedOps* b);

// setup: the stream of the setup work (table uploads, the projector block) at creation and at
// atom moves; each setup ends with a synchronisation of it.
std::unique_ptr<FusedOps> make_fused_ops(const HostGeometry& g, const DevTables<float>& t, int nstates,
                                         DeviceArena& arena, StageProfiler& prof, int* err, cudaStream_t setup);

template <typename T>
inline std::unique_ptr<FusedOps> make_fused_for(const HostGeometry&, const DevTables<T>&, int, DeviceArena&,
                                                StageProfiler&, int*, cudaStream_t) {
  return nullptr;
}
template <>
inline std::unique_ptr<FusedOps> make_fused_for<float>(const HostGeometry& g, const DevTables<float>& t, int n,
                                                       DeviceArena& a, StageProfiler& prof, int* err,
                                                       cudaStream_t setup) {
  return make_fused_ops(g, t, n, a, prof, err, setup);
}

}  // namespace ks
