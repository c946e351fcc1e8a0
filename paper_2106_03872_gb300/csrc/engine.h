// The per-handle engine: device-resident tables, states and work buffers, and the
// operations of the C ABI built from the kernels.  One instance per ks_grid.
#pragma once

#include <memory>

#include "common.h"

namespace ks {

// Device allocation owned by an engine; every allocation is counted for admission.
class DeviceArena {
 public:
  ~DeviceArena();
  void* alloc(size_t bytes);
  size_t bytes() const { return total_; }

 private:
  std::vector<void*> ptrs_;
  size_t total_ = 0;
};

// Device bytes an engine for this cell would hold (used by the serving admission).
size_t engine_device_bytes(const ks_cell_desc& d, int nG, int ncols);

class EngineBase {
 public:
  virtual ~EngineBase() = default;
  virtual const HostGeometry& geo() const = 0;
  virtual int nstates() const = 0;
  virtual ks_precision precision() const = 0;
  virtual size_t device_bytes() const = 0;
  virtual void* states_device() = 0;
  virtual void set_states(const double* c_host, cudaStream_t s) = 0;
  virtual void get_states(double* c_host, cudaStream_t s) = 0;
  virtual void apply_h(const void* psi, void* hpsi, int n, cudaStream_t s) = 0;
  virtual void apply_h_host(const double* psi_host, double* hpsi_host, int n) = 0;
  virtual void density(void* n_out, cudaStream_t s) = 0;
  virtual void orthonormalize(double* S_host, cudaStream_t s) = 0;
  virtual void rayleigh_ritz(double* eig_host, cudaStream_t s) = 0;
  virtual void block_iteration(int niter, double* eig_host, cudaStream_t s) = 0;
  virtual void td_steps(double dt, int nsteps, int propagator, int hartree_xc, double* norm_out,
                        double* energy_out, cudaStream_t s) = 0;
  virtual void randomize_states(uint64_t seed, cudaStream_t s) = 0;
};

std::unique_ptr<EngineBase> make_engine(const ks_cell_desc& d);

}  // namespace ks
