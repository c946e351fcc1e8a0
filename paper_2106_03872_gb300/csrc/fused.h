// Fused mixed-precision (complex64) Hamiltonian path: pruned z-column FFTs, one plane
// kernel per z-plane holding the (x, y) plane in shared memory with the potential and
// the projector add fused between the inverse and forward transforms, and the kinetic
// term fused into the last transform.
#pragma once

#include <memory>

#include "engine.h"
#include "kernels.h"

namespace ks {

class FusedOps {
 public:
  virtual ~FusedOps() = default;
  // hpsi = H psi for n states with potential v (grid order).
  virtual void apply_h(const float2* psi, float2* hpsi, int n, const float* v, cudaStream_t s) = 0;
  // nout = sum_k occ[k] |psi_k(r)|^2 (grid order).
  virtual void density(const float2* psi, int n, const double* occ, float* nout, cudaStream_t s) = 0;
  // out[b][z][x][y] = Omega^{1/2} psi_b(r) on the grid (plane-major: z slowest), the unscaled
  // inverse transform of n packed states, by the pruned z-columns and the in-SMEM y, x passes.
  virtual void real_space(const float2* psi, int n, float2* out, cudaStream_t s) = 0;
  // The atoms moved.  prepare_atoms forms the per-plane projector lists on the host from the
  // geometry's new sphere lists (no device work, so it may overlap kernels in flight);
  // set_atoms uploads them and rebuilds the projector block (t: the engine's re-uploaded
  // tables).  Synchronous.
  virtual void prepare_atoms() = 0;
  virtual void set_atoms(const DevTables<float>& t) = 0;
};

std::unique_ptr<FusedOps> make_fused_ops(const HostGeometry& g, const DevTables<float>& t, int nstates,
                                         DeviceArena& arena, StageProfiler& prof, int* err);

template <typename T>
inline std::unique_ptr<FusedOps> make_fused_for(const HostGeometry&, const DevTables<T>&, int, DeviceArena&,
                                                StageProfiler&, int*) {
  return nullptr;
}
template <>
inline std::unique_ptr<FusedOps> make_fused_for<float>(const HostGeometry& g, const DevTables<float>& t, int n,
                                                       DeviceArena& a, StageProfiler& prof, int* err) {
  return make_fused_ops(g, t, n, a, prof, err);
}

}  // namespace ks
