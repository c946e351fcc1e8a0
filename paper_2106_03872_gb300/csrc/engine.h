// The per-handle engine: device-resident tables, states and work buffers, and the
// operations of the C ABI built from the kernels.  One instance per ks_grid.
#pragma once

#include <map>
#include <memory>
#include <mutex>

#include "common.h"

namespace ks {

// Device memory shared by the engines of a server: slabs obtained with cudaMalloc as the pool
// grows and kept until the pool is destroyed; blocks of 256-byte granularity handed out first
// fit from per-slab free lists and returned without cudaFree.  cudaFree synchronises the whole
// device, so engines that allocate from a pool are created and destroyed without stalling the
// kernels of other engines in flight.  The caller returns a block only once the work that uses
// it has completed (a server synchronises a request's stream before retiring it).  Thread-safe.
class DevicePool {
 public:
  explicit DevicePool(size_t slab_bytes) : slab_bytes_(slab_bytes) {}
  ~DevicePool();
  void* alloc(size_t bytes);
  void free(void* p);
  size_t reserved() const;   // bytes obtained from the device
  size_t in_use() const;     // bytes handed out
  long grows() const;        // slabs obtained (cudaMalloc calls)
  double grow_seconds() const;   // time spent in them

 private:
  struct Slab {
    char* base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_blocks;   // offset -> size, coalesced
  };
  void* take(size_t bytes);   // first fit in the existing slabs (lock held), or null
  size_t slab_bytes_;
  mutable std::mutex mu_;
  std::vector<Slab> slabs_;
  std::map<char*, std::pair<int, size_t>> used_;   // address -> (slab, size)
  size_t reserved_ = 0, in_use_ = 0;
  long grows_ = 0;
  double grow_s_ = 0;
};

// Device allocation owned by an engine; every allocation is counted for admission.  With a pool,
// allocations come from it and go back to it (no cudaMalloc or cudaFree of their own).
class DeviceArena {
 public:
  ~DeviceArena();
  void set_pool(DevicePool* pool) { pool_ = pool; }
  void* alloc(size_t bytes);
  // Frees one allocation of this arena (without a pool the device is synchronised by cudaFree);
  // null is a no-op.
  void release(const void* p);
  size_t bytes() const { return total_; }

 private:
  DevicePool* pool_ = nullptr;
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
  virtual void set_option(int option, int value) = 0;
};

// pool (may be null): the engine's device memory comes from it.
std::unique_ptr<EngineBase> make_engine(const ks_cell_desc& d, DevicePool* pool = nullptr);

// The status a call returns for the tensor-core kernels' error word, read after the call: 0 is
// success; nonzero means a bounded mbarrier wait expired (the kernel recorded it and returned),
// raised as KS_ERR_CUDA with a message.
void raise_tc_status(int flag);

// True when two engines may take their real-time steps together (mixed precision, fused path,
// one grid geometry).
bool td_groupable(const EngineBase* a, const EngineBase* b);
// One ETRS step (Sec. "Real-time propagation"; Hartree and exchange when hartree_xc) of every
// engine in es, in lockstep on stream s: each H application of the step is one packed launch
// over all of them.  norms[i] and energies[i] receive engine i's norm and energy at the start of
// the step.  KS_ERR_ARG unless td_groupable holds for every pair; KS_ERR_DIVERGED on a non-finite
// norm or energy.  Synchronous.
void td_step_engines(const std::vector<EngineBase*>& es, double dt, int hartree_xc, double* norms, double* energies,
                     cudaStream_t s);

}  // namespace ks
