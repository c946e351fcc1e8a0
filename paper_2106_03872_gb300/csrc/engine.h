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
  // Frees one allocation of this arena (the device is synchronised by cudaFree); null is a no-op.
  void release(const void* p);
  size_t bytes() const { return total_; }

 private:
  std::vector<void*> ptrs_;
  std::vector<size_t> sizes_;
  size_t total_ = 0;
};

// Per-stage CUDA-event timing of an engine's kernels (off by default).  Each stage scope
// records an event pair on the launching stream; collect() waits for them and accumulates
// milliseconds and launch counts per stage name.  With the timeline on, every scope is also
// kept as a span (start and end in milliseconds after the first scope recorded since the
// timeline was started), which shows how stages on different streams overlap.
class StageProfiler {
 public:
  struct Entry {
    std::string name;
    double ms = 0;
    long count = 0;
  };
  struct Span {
    int entry;
    double start, end;
  };
  ~StageProfiler();
  void enable(bool on);
  void timeline(bool on);
  bool on() const { return on_; }
  int begin(const char* name, cudaStream_t s);
  void end(int slot, cudaStream_t s);
  void collect();
  const std::vector<Entry>& entries() const { return entries_; }
  const std::vector<Span>& spans() const { return spans_; }
  void reset() {
    collect();
    entries_.clear();
    spans_.clear();
  }

 private:
  struct Pending {
    int entry;
    cudaEvent_t a, b;
  };
  cudaEvent_t get_event();
  bool on_ = false;
  bool timeline_ = false;
  cudaEvent_t base_ = nullptr;
  bool base_set_ = false;
  std::vector<Entry> entries_;
  std::vector<Pending> pending_;
  std::vector<Span> spans_;
  std::vector<cudaEvent_t> free_;
};

class ProfScope {
 public:
  ProfScope(StageProfiler& p, const char* name, cudaStream_t s) : p_(p), s_(s) { slot_ = p_.on() ? p_.begin(name, s) : -1; }
  ~ProfScope() {
    if (slot_ >= 0) p_.end(slot_, s_);
  }

 private:
  StageProfiler& p_;
  cudaStream_t s_;
  int slot_;
};

class EngineBase {
 public:
  StageProfiler prof;
  virtual ~EngineBase() = default;
  virtual const HostGeometry& geo() const = 0;
  virtual int nstates() const = 0;
  virtual ks_precision precision() const = 0;
  virtual size_t device_bytes() const = 0;
  virtual void get_vloc(double* v_host) = 0;
  virtual void* states_device() = 0;
  virtual void set_states(const double* c_host, cudaStream_t s) = 0;
  virtual void get_states(double* c_host, cudaStream_t s) = 0;
  virtual void apply_h(const void* psi, void* hpsi, int n, cudaStream_t s) = 0;
  virtual void apply_h_host(const double* psi_host, double* hpsi_host, int n) = 0;
  virtual void density(void* n_out, cudaStream_t s) = 0;
  virtual void orthonormalize(double* S_host, cudaStream_t s) = 0;
  virtual void rayleigh_ritz(double* eig_host, cudaStream_t s) = 0;
  virtual void block_iteration(int niter, double* eig_host, cudaStream_t s) = 0;
  virtual void block_iteration_teter(int niter, double* eig_host, cudaStream_t s) = 0;
  virtual void scf(int max_iter, int eig_iters, int mixer, double mix, int history, double tol, double* eig_out,
                   double* resid_out, int* iters_done, cudaStream_t s) = 0;
  virtual void td_steps(double dt, int nsteps, int propagator, int hartree_xc, double* norm_out,
                        double* energy_out, double* dipole_out, cudaStream_t s) = 0;
  virtual void kick(const double kappa[3], cudaStream_t s) = 0;
  virtual void dipole(double* d_host, cudaStream_t s) = 0;
  virtual void forces(double* f_host, cudaStream_t s) = 0;
  virtual void set_positions(const double* pos, cudaStream_t s) = 0;
  virtual void ehrenfest(double dt, int nsteps, int hartree_xc, const double* mass, double* vel, double* pos_out,
                         double* energy_out, cudaStream_t s) = 0;
  virtual void randomize_states(uint64_t seed, cudaStream_t s) = 0;
};

std::unique_ptr<EngineBase> make_engine(const ks_cell_desc& d);

}  // namespace ks
