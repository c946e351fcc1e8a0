// Engine<T>: the device-resident state of one cell and the operations of the C ABI,
// composed from the kernels.  T = double is the FP64 path; T = float the mixed path
// (its fused Hamiltonian lives in fused.cu and plugs in through FusedOps).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <functional>
#include <cstring>
#include <type_traits>

#include "engine.h"
#include "fused.h"
#include "kernels.h"

namespace ks {

DevicePool::~DevicePool() {
  for (auto& sl : slabs_) cudaFree(sl.base);
}

// First fit in the slabs; a new slab when none has room.  The slab is obtained from the device
// without the lock held (cudaMalloc of a slab can take tens of milliseconds on a busy device,
// and every other engine's allocations and releases would wait behind it).
void* DevicePool::alloc(size_t bytes) {
  bytes = std::max<size_t>(256, (bytes + 255) / 256 * 256);
  std::unique_lock<std::mutex> lk(mu_);
  if (void* p = take(bytes)) return p;
  lk.unlock();
  Slab sl;
  sl.size = std::max(slab_bytes_, bytes);
  void* base = nullptr;
  const auto g0 = std::chrono::steady_clock::now();
  const cudaError_t e = cudaMalloc(&base, sl.size);
  const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - g0).count();
  lk.lock();
  grow_s_ += dt;
  ++grows_;
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (void* p = take(bytes)) return p;                             // another thread's slab may fit
    fail(KS_ERR_NOMEM, "device pool: cudaMalloc of a %zu-byte slab failed (%s)", sl.size, cudaGetErrorString(e));
  }
  sl.base = static_cast<char*>(base);
  sl.free_blocks[0] = sl.size;
  slabs_.push_back(std::move(sl));
  reserved_ += slabs_.back().size;
  void* p = take(bytes);
  if (!p) fail(KS_ERR_STATE, "internal: device pool slab without room");
  return p;
}

// A block of `bytes` from the first slab with a free block that large (lock held), or null.
void* DevicePool::take(size_t bytes) {
  for (int si = 0; si < (int)slabs_.size(); ++si) {
    Slab& sl = slabs_[si];
    for (auto it = sl.free_blocks.begin(); it != sl.free_blocks.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, size = it->second;
      sl.free_blocks.erase(it);
      if (size > bytes) sl.free_blocks[off + bytes] = size - bytes;
      char* p = sl.base + off;
      used_[p] = {si, bytes};
      in_use_ += bytes;
      return p;
    }
  }
  return nullptr;
}

void DevicePool::free(void* vp) {
  if (!vp) return;
  std::lock_guard<std::mutex> lk(mu_);
  auto it = used_.find(static_cast<char*>(vp));
  if (it == used_.end()) fail(KS_ERR_STATE, "internal: device pool release of an unknown block");
  Slab& sl = slabs_[it->second.first];
  size_t off = static_cast<size_t>(it->first - sl.base), size = it->second.second;
  in_use_ -= size;
  used_.erase(it);
  // coalesce with the free neighbours inside the slab
  auto next = sl.free_blocks.lower_bound(off);
  if (next != sl.free_blocks.end() && next->first == off + size) {
    size += next->second;
    next = sl.free_blocks.erase(next);
  }
  if (next != sl.free_blocks.begin()) {
    auto prev = std::prev(next);
    if (prev->first + prev->second == off) {
      prev->second += size;
      return;
    }
  }
  sl.free_blocks[off] = size;
}

size_t DevicePool::reserved() const {
  std::lock_guard<std::mutex> lk(mu_);
  return reserved_;
}

size_t DevicePool::in_use() const {
  std::lock_guard<std::mutex> lk(mu_);
  return in_use_;
}

long DevicePool::grows() const {
  std::lock_guard<std::mutex> lk(mu_);
  return grows_;
}

double DevicePool::grow_seconds() const {
  std::lock_guard<std::mutex> lk(mu_);
  return grow_s_;
}

DeviceArena::~DeviceArena() {
  for (void* p : ptrs_) {
    if (pool_)
      pool_->free(p);
    else
      cudaFree(p);
  }
}

void* DeviceArena::alloc(size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) / 256 * 256;
  if (pool_)
    p = pool_->alloc(bytes);
  else
    KS_CUDA(cudaMalloc(&p, bytes));
  ptrs_.push_back(p);
  sizes_.push_back(bytes);
  total_ += bytes;
  return p;
}

void DeviceArena::release(const void* p) {
  if (!p) return;
  for (size_t i = 0; i < ptrs_.size(); ++i)
    if (ptrs_[i] == p) {
      if (pool_)
        pool_->free(ptrs_[i]);
      else
        KS_CUDA(cudaFree(ptrs_[i]));
      total_ -= sizes_[i];
      ptrs_.erase(ptrs_.begin() + i);
      sizes_.erase(sizes_.begin() + i);
      return;
    }
  fail(KS_ERR_STATE, "internal: release of a pointer the arena does not own");
}

StageProfiler::~StageProfiler() {
  for (auto& p : pending_) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : free_) cudaEventDestroy(e);
  if (base_) cudaEventDestroy(base_);
}

void StageProfiler::enable(bool on) {
  if (!on) collect();
  on_ = on;
}

void StageProfiler::timeline(bool on) {
  collect();
  timeline_ = on;
  base_set_ = false;
  spans_.clear();
  if (on && !base_) KS_CUDA(cudaEventCreate(&base_));
}

cudaEvent_t StageProfiler::get_event() {
  if (!free_.empty()) {
    cudaEvent_t e = free_.back();
    free_.pop_back();
    return e;
  }
  cudaEvent_t e;
  KS_CUDA(cudaEventCreate(&e));
  return e;
}

int StageProfiler::begin(const char* name, cudaStream_t s) {
  int idx = -1;
  for (size_t i = 0; i < entries_.size(); ++i)
    if (entries_[i].name == name) idx = (int)i;
  if (idx < 0) {
    entries_.push_back(Entry{name, 0.0, 0});
    idx = (int)entries_.size() - 1;
  }
  Pending p{idx, get_event(), get_event()};
  if (timeline_ && !base_set_) {
    KS_CUDA(cudaEventRecord(base_, s));
    base_set_ = true;
  }
  KS_CUDA(cudaEventRecord(p.a, s));
  pending_.push_back(p);
  return (int)pending_.size() - 1;
}

void StageProfiler::end(int slot, cudaStream_t s) { KS_CUDA(cudaEventRecord(pending_[slot].b, s)); }

void StageProfiler::collect() {
  for (auto& p : pending_) {
    KS_CUDA(cudaEventSynchronize(p.b));
    float ms = 0;
    KS_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
    entries_[p.entry].ms += ms;
    entries_[p.entry].count += 1;
    if (timeline_ && base_set_) {
      float t0 = 0, t1 = 0;
      KS_CUDA(cudaEventElapsedTime(&t0, base_, p.a));
      KS_CUDA(cudaEventElapsedTime(&t1, base_, p.b));
      spans_.push_back(Span{p.entry, t0, t1});
    }
    free_.push_back(p.a);
    free_.push_back(p.b);
  }
  pending_.clear();
}

namespace {

constexpr int MAX_STEPS_CHUNK = 1024;
constexpr size_t GRID_BUDGET = size_t(1) << 30;   // full-grid work buffer of the plain path

template <typename T> size_t full_grid_batch(int N, int ns) {
  const size_t per = (size_t)N * N * N * sizeof(cplx<T>);
  size_t b = std::max<size_t>(1, GRID_BUDGET / per);
  return std::min<size_t>(b, (size_t)ns);
}

template <typename T> class Engine final : public EngineBase {
 public:
  using C = cplx<T>;

  explicit Engine(const ks_cell_desc& d, DevicePool* pool = nullptr) : prec_(d.prec), ns_(d.nstates) {
    arena_.set_pool(pool);
    build_geometry(d, g_);                                            // validates the cell (KS_ERR_ARG)
    // side stream (highest priority, non-blocking): the CholQR factor that overlaps H psi, and
    // the setup work here and at atom moves (table uploads, V_loc, the projector block), which
    // so neither waits behind other engines' kernels nor serialises on the legacy stream
    int lo = 0, hi = 0;
    KS_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    KS_CUDA(cudaStreamCreateWithPriority(&aux_, cudaStreamNonBlocking, hi));
    setup_ = aux_;
    const int N = g_.N, nG = g_.nG;
    const size_t N3 = (size_t)N * N * N;
    const size_t sn = (size_t)ns_ * nG;
    // ---- tables
    t_.N = N;
    t_.nG = nG;
    t_.ncols = g_.ncols;
    t_.natoms = g_.natoms;
    t_.nproj = g_.nproj;
    t_.ncov = (int)g_.cov_idx.size();
    t_.xr = g_.xr;
    t_.L = g_.L;
    t_.omega = g_.omega;
    t_.dV = g_.dV;
    t_.D = g_.D;
    t_.gidx = upload(g_.gidx);
    t_.g2half = upload_real(g_.g2half);
    std::vector<T> tw(2 * N);
    for (int i = 0; i < 2 * N; ++i) tw[i] = (T)g_.tw[i];
    t_.tw = reinterpret_cast<const C*>(upload(tw));
    t_.col_xy = upload(g_.col_xy);
    t_.col_off = upload(g_.col_off);
    t_.col_half = upload(g_.col_half);
    t_.sph_off = upload(g_.sph_off);
    t_.sph_idx = upload(g_.sph_idx);
    t_.sph_atom = upload(g_.sph_atom);
    t_.sph_beta = upload_real(g_.sph_beta);
    t_.sph_zorder = upload(g_.sph_zorder);
    t_.cov_idx = upload(g_.cov_idx);
    t_.cov_off = upload(g_.cov_off);
    t_.cov_ent = upload(g_.cov_ent);
    vloc_ = alloc<T>(N3);
    vloc64_ = alloc<double>(N3);
    vmm_ = alloc<double>(2);
    vtot_ = alloc<T>(N3);
    occ_ = const_cast<double*>(upload(g_.occ));
    // ---- states: 6 buffers (resident psi, H psi, and 4 work buffers for the real-time step)
    for (int i = 0; i < 6; ++i) {
      buf_[i] = alloc<C>(sn);
      KS_CUDA(cudaMemsetAsync(buf_[i], 0, sn * sizeof(C), setup_));
    }
    psi_ = buf_[0];
    hpsi_ = buf_[1];
    staging_ = alloc<double2>(sn);
    // ---- Hamiltonian work
    status_ = alloc<int>(4);
    KS_CUDA(cudaMemsetAsync(status_, 0, 4 * sizeof(int), setup_));
    fused_ = make_fused_for(g_, t_, ns_, arena_, prof, status_ + 1, setup_);
    if (!fused_) {
      batch_ = (int)full_grid_batch<T>(N, ns_);
      grid_ = alloc<C>((size_t)batch_ * N3);
      proj_ = alloc<C>((size_t)batch_ * std::max(1, g_.natoms) * g_.nproj);
    }
    // ---- dense LA
    const size_t nn = (size_t)ns_ * ns_;
    part_elems_ = std::max<size_t>(nn * 8, 4096);
    if (use_tc()) {
      part_elems_ = std::max(part_elems_, tc_overlap_part_elems(ns_, ns_));
      rotws_bytes_ = tc_rotation_workspace_bytes(ns_, 2 * ns_);
      rotws_ = arena_.alloc(rotws_bytes_);
    }
    part_ = alloc<double2>(part_elems_);
    mS_ = alloc<double2>(nn);
    mA_ = alloc<double2>(nn);
    mM_ = alloc<double2>(nn);
    mV_ = alloc<double2>(nn);
    mT_ = alloc<double2>(nn);
    mC_ = alloc<double2>(nn);
    mF_ = alloc<double2>(nn);
    mCat_ = alloc<double2>(2 * nn);
    eig_ = alloc<double>(ns_);
    lam_ = alloc<double>(ns_);
    if (mixed_cholesky()) chw_ = alloc<double2>(cholesky_mixed_workspace(ns_));
    if (fused_rr()) {
      hraw32_ = alloc<float2>(nn);
      m32_ = alloc<float2>(nn);
      mcat32_ = alloc<float2>(2 * nn);
      aexp_ = alloc<float2>(nn);
      vexp_ = alloc<float2>(nn);
      perm_ = alloc<int>(ns_);
    }
    // ---- potentials / real-time
    dens_ = alloc<T>(N3);
    pwork_ = alloc<C>(N3);
    hxc_partials_ = alloc<double>(HXC_BLOCKS * 3);
    nin_ = alloc<T>(N3);
    resid_dev_ = alloc<double>(1);
    dip_partials_ = alloc<double>(HXC_BLOCKS * 3);
    trr_ = alloc<double2>(ns_);
    dipoles_dev_ = alloc<double>(3 * MAX_STEPS_CHUNK);
    parts_ = alloc<double>(4);
    dots_ = alloc<double2>(ns_);
    norms_dev_ = alloc<double>(MAX_STEPS_CHUNK);
    energies_dev_ = alloc<double>(MAX_STEPS_CHUNK);
    KS_CUDA(cudaEventCreateWithFlags(&ev_gram_, cudaEventDisableTiming));
    KS_CUDA(cudaEventCreateWithFlags(&ev_hraw_, cudaEventDisableTiming));
    KS_CUDA(cudaEventCreateWithFlags(&ev_chol_, cudaEventDisableTiming));
    KS_CUDA(cudaEventCreateWithFlags(&ev_ritz_, cudaEventDisableTiming));
    update_vloc(setup_);                                             // ends with a synchronisation
  }

  ~Engine() override {
    if (aux_) {
      cudaStreamSynchronize(aux_);
      cudaStreamDestroy(aux_);
    }
    if (ev_gram_) cudaEventDestroy(ev_gram_);
    if (ev_hraw_) cudaEventDestroy(ev_hraw_);
    if (ev_chol_) cudaEventDestroy(ev_chol_);
    if (ev_ritz_) cudaEventDestroy(ev_ritz_);
  }

  const HostGeometry& geo() const override { return g_; }
  int nstates() const override { return ns_; }
  ks_precision precision() const override { return prec_; }
  size_t device_bytes() const override { return arena_.bytes(); }
  void* states_device() override {
    hpsi_valid_ = false;   // the caller may write the block
    return psi_;
  }

  void set_states(const double* c_host, cudaStream_t s) override {
    const size_t sn = (size_t)ns_ * g_.nG;
    KS_CUDA(cudaMemcpyAsync(staging_, c_host, sn * sizeof(double2), cudaMemcpyHostToDevice, s));
    from_c128<T>(staging_, psi_, sn, s);
    hpsi_valid_ = false;
    KS_CUDA(cudaStreamSynchronize(s));
  }

  void get_states(double* c_host, cudaStream_t s) override {
    const size_t sn = (size_t)ns_ * g_.nG;
    to_c128<T>(psi_, staging_, sn, s);
    KS_CUDA(cudaMemcpyAsync(c_host, staging_, sn * sizeof(double2), cudaMemcpyDeviceToHost, s));
    KS_CUDA(cudaStreamSynchronize(s));
  }

  // Pieces of td_steps for a lockstep group (td_step_engines): the potential reset before the
  // step, the asynchronous read of slot 0's norm and energy, and the buffer roles after it.
  bool groupable_with(const Engine& o) const {
    return fused_ && o.fused_ && fused_same_geometry(fused_.get(), o.fused_.get());
  }
  void td_prepare(int hartree_xc, cudaStream_t s) {
    hpsi_valid_ = false;
    if (!hartree_xc)
      KS_CUDA(cudaMemcpyAsync(vtot_, vloc_, (size_t)g_.N * g_.N * g_.N * sizeof(T), cudaMemcpyDeviceToDevice, s));
  }
  void td_read_slot0(double* nrm, double* e, cudaStream_t s) {
    KS_CUDA(cudaMemcpyAsync(nrm, norms_dev_, sizeof(double), cudaMemcpyDeviceToHost, s));
    KS_CUDA(cudaMemcpyAsync(e, energies_dev_, sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  void td_finish(cudaStream_t s) {
    check_tc_status(s);
    if (hpsi_ == psi_) hpsi_ = spare(psi_, nullptr);
  }

  void set_option(int option, int value) override {
    if (option == KS_OPT_FP64_SUBSPACE) {
      if (value != 0 && value != 1) fail(KS_ERR_ARG, "KS_OPT_FP64_SUBSPACE takes 0 or 1, got %d", value);
      if (sizeof(T) == 8) return;                                     // the FP64 path has it always
      fp64_subspace_ = value != 0;
      hpsi_valid_ = false;
      return;
    }
    fail(KS_ERR_ARG, "unknown option %d", option);
  }

  void randomize_states(uint64_t seed, cudaStream_t s) override {
    random_states<T>(psi_, (size_t)ns_ * g_.nG, seed, s);
    hpsi_valid_ = false;
  }

  // ------------------------------------------------------------------------------------------
  // H psi (Eq. 2): G -> r, V psi + V_NL psi on the grid, r -> G, keep S, + |G|^2/2 c.
  // ------------------------------------------------------------------------------------------
  void apply_h(const void* psi_v, void* hpsi_v, int n, cudaStream_t s) override {
    const C* psi = static_cast<const C*>(psi_v);
    C* hpsi = static_cast<C*>(hpsi_v);
    if (n < 0 || n > ns_) fail(KS_ERR_ARG, "apply_h: nstates=%d outside [0, %d]", n, ns_);
    if (n == 0) return;
    ProfScope scope(prof, "apply_h", s);
    if constexpr (std::is_same<T, float>::value) {
      if (fused_) {
        fused_->apply_h(psi, hpsi, n, vtot_, s);
        return;
      }
    }
    const int N = g_.N;
    const size_t N3 = (size_t)N * N * N;
    const T rs = T(1.0 / std::sqrt(g_.omega));
    for (int b0 = 0; b0 < n; b0 += batch_) {
      const int nb = std::min(batch_, n - b0);
      const C* in = psi + (size_t)b0 * g_.nG;
      KS_CUDA(cudaMemsetAsync(grid_, 0, (size_t)nb * N3 * sizeof(C), s));
      scatter_sphere<T>(in, grid_, t_, nb, s);
      {
        ProfScope f(prof, "fft_lines", s);
        for (int ax = 2; ax >= 0; --ax) fft_axis<T>(grid_, nb, N, ax, +1, t_.tw, s);
      }
      // grid holds psi' = Omega^{1/2} psi.  p = dV sum beta psi = dV Omega^{-1/2} sum beta psi'.
      nl_project<T>(grid_, t_, proj_, nb, T(g_.dV) * rs, s);
      multiply_potential<T>(grid_, vtot_, (int)N3, nb, s);
      // u' = Omega^{1/2} u: add Omega^{1/2} D beta p
      nl_add<T>(grid_, t_, proj_, nb, T(g_.D * std::sqrt(g_.omega)), s);
      {
        ProfScope f(prof, "fft_lines", s);
        for (int ax = 0; ax < 3; ++ax) fft_axis<T>(grid_, nb, N, ax, -1, t_.tw, s);
      }
      gather_kinetic<T>(grid_, in, hpsi + (size_t)b0 * g_.nG, t_, nb, T(1.0 / double(N3)), s);
    }
  }

  void apply_h_host(const double* psi_host, double* hpsi_host, int n) override {
    if (n < 0 || n > ns_) fail(KS_ERR_ARG, "apply_h_host: nstates=%d outside [0, %d]", n, ns_);
    cudaStream_t s = 0;
    const size_t sn = (size_t)n * g_.nG;
    C* in = spare(psi_, hpsi_);
    C* out = spare3(psi_, hpsi_, in);
    KS_CUDA(cudaMemcpyAsync(staging_, psi_host, sn * sizeof(double2), cudaMemcpyHostToDevice, s));
    from_c128<T>(staging_, in, sn, s);
    apply_h(in, out, n, s);
    to_c128<T>(out, staging_, sn, s);
    KS_CUDA(cudaMemcpyAsync(hpsi_host, staging_, sn * sizeof(double2), cudaMemcpyDeviceToHost, s));
    check_tc_status(s);
  }

  // ------------------------------------------------------------------------------------------
  // Density (Eq. 1) of n states of `psi`, into nout [N^3] (grid order), fixed state order.
  // ------------------------------------------------------------------------------------------
  void density_of(const C* psi, int n, T* nout, cudaStream_t s) {
    ProfScope scope(prof, "density", s);
    if constexpr (std::is_same<T, float>::value) {
      if (fused_) {
        fused_->density(psi, n, occ_, nout, s);
        return;
      }
    }
    const int N = g_.N;
    const size_t N3 = (size_t)N * N * N;
    const T scale = T(1.0 / g_.omega);
    for (int b0 = 0; b0 < n; b0 += batch_) {
      const int nb = std::min(batch_, n - b0);
      KS_CUDA(cudaMemsetAsync(grid_, 0, (size_t)nb * N3 * sizeof(C), s));
      scatter_sphere<T>(psi + (size_t)b0 * g_.nG, grid_, t_, nb, s);
      for (int ax = 2; ax >= 0; --ax) fft_axis<T>(grid_, nb, N, ax, +1, t_.tw, s);
      density_accumulate<T>(grid_, occ_ + b0, nout, (int)N3, nb, scale, b0 == 0, s);
    }
  }

  void density(void* n_out, cudaStream_t s) override { density_of(psi_, ns_, static_cast<T*>(n_out), s); }

  // V = V_loc + v_H[n] + v_x[n] (periodic Poisson in Fourier space, v_H(G=0) = 0; Slater exchange)
  void update_potential(const T* n, cudaStream_t s) {
    ProfScope scope(prof, "hartree_xc", s);
    const int N = g_.N;
    const size_t N3 = (size_t)N * N * N;
    real_to_complex<T>(n, pwork_, (int)N3, s);
    for (int ax = 2; ax >= 0; --ax) fft_axis<T>(pwork_, 1, N, ax, -1, t_.tw, s);
    poisson_multiply<T>(pwork_, N, g_.L, T(1.0 / double(N3)), s);
    for (int ax = 0; ax < 3; ++ax) fft_axis<T>(pwork_, 1, N, ax, +1, t_.tw, s);
    hxc_combine<T>(n, pwork_, vloc_, vtot_, hxc_partials_, (int)N3, HXC_BLOCKS, s);
    hxc_finish(hxc_partials_, HXC_BLOCKS, g_.dV, parts_, s);
  }

  // ------------------------------------------------------------------------------------------
  // CholQR: S = Psi^H Psi, S = L L^H, Psi <- Psi L^{-H}  (rows: psi <- conj(L^{-1}) psi)
  // ------------------------------------------------------------------------------------------
  // M = conj(L^{-1}) for S = L L^H (mS_ -> mM_), on stream st
  // With m32 (the fused block iteration, which reads only the FP32 copy), the single FP32
  // pass of the mixed path without its FP64 refinement.
  void factor(cudaStream_t st, float2* m32 = nullptr) {
    const int n = ns_;
    ProfScope p(prof, "cholesky", st);
    if (mixed_cholesky() && !fp64_subspace_) {
      cholesky_inverse_mixed(mS_, mM_, n, 1e-6, chw_, status_, st, m32, m32 == nullptr);
    } else {
      KS_CUDA(cudaMemcpyAsync(mF_, mS_, (size_t)n * n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
      cholesky_inverse_tol(mF_, mM_, n, sizeof(T) == 8 ? 1e-12 : 1e-6, status_, st);
    }
  }

  void cholqr_factor(cudaStream_t s) {
    {
      ProfScope p(prof, "gram", s);
      overlap(psi_, psi_, ns_, mS_, s);
      hermitize(mS_, ns_, s);
    }
    factor(s);
  }

  void cholqr_rotate(cudaStream_t s) {
    C* out = spare(psi_, hpsi_);
    {
      ProfScope p(prof, "rotate", s);
      rot(mM_, psi_, out, s);
    }
    swap_in(psi_, out);
  }

  // The public call reads the status before rotating, so a failure leaves the states as they
  // were on every precision path.
  void orthonormalize(double* S_host, cudaStream_t s) override {
    hpsi_valid_ = false;
    KS_CUDA(cudaMemsetAsync(status_, 0, sizeof(int), s));
    cholqr_factor(s);
    int st = 0;
    KS_CUDA(cudaMemcpyAsync(&st, status_, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (S_host) KS_CUDA(cudaMemcpyAsync(S_host, mS_, (size_t)ns_ * ns_ * sizeof(double2), cudaMemcpyDeviceToHost, s));
    KS_CUDA(cudaStreamSynchronize(s));
    check_tc_status(s);
    if (st) fail(KS_ERR_NOT_POSDEF, "CholQR: Gram matrix not positive definite at column %d", st - 1);
    cholqr_rotate(s);
    KS_CUDA(cudaStreamSynchronize(s));
    check_tc_status(s);
  }

  // Rayleigh-Ritz on (psi_, hpsi_): H_sub = Psi^H H Psi, eigh, rotate both.
  void rr_core(cudaStream_t s) {
    const int n = ns_;
    {
      ProfScope p(prof, "gram", s);
      overlap(psi_, hpsi_, n, mA_, s);
      hermitize(mA_, n, s);
    }
    {
      ProfScope p(prof, "eigh", s);
      eigh_sub(n, mM_, s);
    }
    ProfScope p(prof, "rotate", s);
    C* o1 = spare(psi_, hpsi_);
    rot(mM_, psi_, o1, s);
    swap_in(psi_, o1);
    C* o2 = spare(psi_, hpsi_);
    rot(mM_, hpsi_, o2, s);
    swap_in(hpsi_, o2);
  }

  void rayleigh_ritz(double* eig_host, cudaStream_t s) override {
    hpsi_valid_ = false;
    apply_h(psi_, hpsi_, ns_, s);
    rr_core(s);
    if (eig_host) KS_CUDA(cudaMemcpyAsync(eig_host, eig_, ns_ * sizeof(double), cudaMemcpyDeviceToHost, s));
    check_tc_status(s);
  }

  void block_iteration(int niter, double* eig_host, cudaStream_t s) override {
    if (niter < 0) fail(KS_ERR_ARG, "niter=%d", niter);
    const double alpha = 1.0 / (g_.ecut + (g_.vmax - g_.vmin) + g_.D);
    KS_CUDA(cudaMemsetAsync(status_, 0, sizeof(int), s));
    // Per iteration (Sec. Ground-state solution): CholQR, H psi, Rayleigh-Ritz, SD update,
    // reorganised around the linearity of H:
    //  - S = psi^H psi and H_raw = psi^H (H psi) are formed on the raw block; the factor M of S,
    //    H_sub = conj(M) H_raw M^T, its eigenvectors Vt, C = Vt M and the step matrix
    //    Mcat = [(I + alpha Lambda) C | -alpha C] run on the side stream (one SM), while
    //  - the main stream applies H to H psi (H^2 psi);
    //  - then psi <- Mcat [psi; H psi] and H psi <- Mcat [H psi; H^2 psi].
    // On the bf16x3 path with n <= 128 the side stream's Rayleigh-Ritz step is one CTA
    // (rr_step_mixed: subspace matrix, eigenpairs, C and Mcat in FP32, rows in ascending order
    // of the FP32 eigenvalues); the reported FP64 Rayleigh quotients follow on the side
    // stream while the main stream rotates.
    // H psi enters the next iteration without a new application of H to psi; it is recomputed
    // directly on entry to a call whose block changed and every HPSI_REFRESH iterations.
    const int n = ns_;
    const bool mixed = sizeof(T) == 4;
    const bool frr = fused_rr() && !fp64_subspace_;
    const bool mixed_sub = mixed && !fp64_subspace_;     // FP32 subspace products and eigensolver
    bool ritz_pending = false;
    for (int it = 0; it < niter; ++it) {
      if (!hpsi_valid_ || hpsi_age_ >= HPSI_REFRESH) {
        apply_h(psi_, hpsi_, n, s);
        hpsi_age_ = 0;
      }
      {
        ProfScope p(prof, "gram", s);
        overlap(psi_, psi_, n, mS_, s);
        hermitize(mS_, n, s);
      }
      KS_CUDA(cudaEventRecord(ev_gram_, s));
      {
        ProfScope p(prof, "gram", s);
        overlap(psi_, hpsi_, n, mA_, s, frr ? hraw32_ : nullptr);
      }
      KS_CUDA(cudaEventRecord(ev_hraw_, s));
      // side stream: factor, subspace matrix, eigenpairs, step matrix
      KS_CUDA(cudaStreamWaitEvent(aux_, ev_gram_, 0));
      factor(aux_, frr ? m32_ : nullptr);
      KS_CUDA(cudaStreamWaitEvent(aux_, ev_hraw_, 0));
      if (frr) {
        {
          ProfScope p(prof, "rr_step", aux_);
          rr_step_mixed(hraw32_, m32_, alpha, n, mcat32_, aexp_, vexp_, perm_, aux_);
        }
        {
          ProfScope p(prof, "rot_prep", aux_);
          tc_rotate_prepare(mcat32_, n, 2 * n, rotws_, rotws_bytes_, aux_);
        }
        KS_CUDA(cudaEventRecord(ev_chol_, aux_));
        // the reported eigenvalues, while the main stream rotates
        {
          ProfScope p(prof, "ritz_values", aux_);
          ritz_values(aexp_, vexp_, perm_, n, eig_, aux_);
        }
        KS_CUDA(cudaEventRecord(ev_ritz_, aux_));
        ritz_pending = true;
      } else {
        {
          ProfScope p(prof, "subspace", aux_);
          small_product(mA_, mM_, n, SP_TRANS_B, mixed_sub, mT_, aux_);   // H_raw M^T
          small_product(mM_, mT_, n, SP_CONJ_A, mixed_sub, mA_, aux_);    // conj(M) H_raw M^T
          hermitize(mA_, n, aux_);
        }
        {
          ProfScope p(prof, "eigh", aux_);
          eigh_sub(n, mT_, aux_);
        }
        {
          ProfScope p(prof, "subspace", aux_);
          small_product(mT_, mM_, n, 0, mixed_sub, mC_, aux_);        // C = Vt M
          sd_matrix(mC_, eig_, alpha, n, mCat_, aux_);
        }
        KS_CUDA(cudaEventRecord(ev_chol_, aux_));
      }
      // main stream: H^2 psi meanwhile
      C* h2 = spare(psi_, hpsi_);
      apply_h(hpsi_, h2, n, s);
      KS_CUDA(cudaStreamWaitEvent(s, ev_chol_, 0));
      {
        ProfScope p(prof, "rotate", s);
        C* o1 = spare3(psi_, hpsi_, h2);
        C* o2 = spare4(psi_, hpsi_, h2, o1);
        if (frr) {
          rot_prepared(psi_, hpsi_, o1, s);
          rot_prepared(hpsi_, h2, o2, s);
        } else {
          rot(mCat_, psi_, o1, s, hpsi_);
          rot(mCat_, hpsi_, o2, s, h2);
        }
        psi_ = o1;
        hpsi_ = o2;
      }
      hpsi_valid_ = true;
      ++hpsi_age_;
    }
    if (ritz_pending) KS_CUDA(cudaStreamWaitEvent(s, ev_ritz_, 0));
    int st = 0;
    KS_CUDA(cudaMemcpyAsync(&st, status_, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (eig_host) KS_CUDA(cudaMemcpyAsync(eig_host, eig_, ns_ * sizeof(double), cudaMemcpyDeviceToHost, s));
    KS_CUDA(cudaStreamSynchronize(s));
    check_tc_status(s);
    if (st) fail(KS_ERR_NOT_POSDEF, "block iteration: Gram matrix not positive definite at column %d", st - 1);
  }

  // ------------------------------------------------------------------------------------------
  // Teter-preconditioned steepest descent (Sec. Ground-state solution).  The preconditioner
  // scales every state per G, so H psi of the update is no rotation of [H psi; H^2 psi]: each
  // iteration runs CholQR, H psi, Rayleigh-Ritz and the update in order.
  // ------------------------------------------------------------------------------------------
  void block_iteration_teter(int niter, double* eig_host, cudaStream_t s) override {
    if (niter < 0) fail(KS_ERR_ARG, "niter=%d", niter);
    hpsi_valid_ = false;
    const double shift = (g_.vmax - g_.vmin) + g_.D;
    const double tmin = 0.5 * (2.0 * M_PI / g_.L) * (2.0 * M_PI / g_.L);   // smallest nonzero |G|^2 / 2
    KS_CUDA(cudaMemsetAsync(status_, 0, sizeof(int), s));
    for (int it = 0; it < niter; ++it) {
      cholqr_factor(s);
      cholqr_rotate(s);
      apply_h(psi_, hpsi_, ns_, s);
      rr_core(s);
      ProfScope p(prof, "teter_update", s);
      teter_update<T>(psi_, hpsi_, t_.g2half, eig_, trr_, shift, tmin, g_.nG, ns_, s);
    }
    int st = 0;
    KS_CUDA(cudaMemcpyAsync(&st, status_, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (eig_host) KS_CUDA(cudaMemcpyAsync(eig_host, eig_, ns_ * sizeof(double), cudaMemcpyDeviceToHost, s));
    KS_CUDA(cudaStreamSynchronize(s));
    check_tc_status(s);
    if (st) fail(KS_ERR_NOT_POSDEF, "preconditioned block iteration: Gram matrix not positive definite at column %d",
                 st - 1);
  }

  // ------------------------------------------------------------------------------------------
  // Self-consistent field (Sec. Ground-state solution) with static linear mixing.
  // ------------------------------------------------------------------------------------------
  void scf(int max_iter, int eig_iters, int mixer, double mix, int history, double tol, double* eig_out,
           double* resid_out, int* iters_done, cudaStream_t s) override {
    if (max_iter < 0 || eig_iters < 1 || mixer < 0 || mixer > 2 || !(mix > 0.0 && mix <= 1.0) || history < 1 ||
        history > PULAY_MAX || !(tol >= 0.0))
      fail(KS_ERR_ARG, "scf: max_iter=%d eig_iters=%d mixer=%d mix=%g history=%d tol=%g", max_iter, eig_iters, mixer,
           mix, history, tol);
    const int N3 = g_.N * g_.N * g_.N;
    if (mixer != 0 && !hist_n_[0]) {
      for (int i = 0; i < PULAY_MAX; ++i) {
        hist_n_[i] = alloc<T>(N3);
        hist_r_[i] = alloc<T>(N3);
      }
      pulay_partials_ = alloc<double>((size_t)HXC_BLOCKS * (2 + PULAY_MAX));
      pulay_out_ = alloc<double>(2 + PULAY_MAX);
    }
    std::vector<double> eig(ns_);
    std::vector<double> A((size_t)PULAY_MAX * PULAY_MAX, 0.0);   // <R_i|R_j> of the history slots
    std::vector<int> order;                                       // slots, oldest first
    orthonormalize(nullptr, s);
    density_of(psi_, ns_, nin_, s);
    int it = 0;
    for (; it < max_iter; ++it) {
      update_potential(nin_, s);
      hpsi_valid_ = false;
      block_iteration(eig_iters, eig.data(), s);
      orthonormalize(nullptr, s);
      density_of(psi_, ns_, dens_, s);
      double r = 0.0;
      if (mixer == 0) {
        ProfScope p(prof, "density_mix", s);
        density_mix<T>(dens_, nin_, N3, mix, hxc_partials_, HXC_BLOCKS, s);
        sum_partials(hxc_partials_, HXC_BLOCKS, g_.dV, resid_dev_, s);
        KS_CUDA(cudaMemcpyAsync(&r, resid_dev_, sizeof(double), cudaMemcpyDeviceToHost, s));
        KS_CUDA(cudaStreamSynchronize(s));
      } else {
        ProfScope p(prof, "density_mix", s);
        // the new pair goes to the oldest slot once the history is full
        if ((int)order.size() == history) order.erase(order.begin());
        int slot = 0;
        while (std::find(order.begin(), order.end(), slot) != order.end()) ++slot;
        PulayRefs<T> refs{};
        refs.m = (int)order.size();
        for (int q = 0; q < refs.m; ++q) refs.r[q] = hist_r_[order[q]];
        double out[2 + PULAY_MAX];
        pulay_store<T>(dens_, nin_, hist_n_[slot], hist_r_[slot], N3, refs, pulay_partials_, HXC_BLOCKS, g_.dV,
                       pulay_out_, s);
        KS_CUDA(cudaMemcpyAsync(out, pulay_out_, sizeof(out), cudaMemcpyDeviceToHost, s));
        KS_CUDA(cudaStreamSynchronize(s));
        r = out[0];
        A[slot * PULAY_MAX + slot] = out[1];
        for (int q = 0; q < refs.m; ++q) {
          A[slot * PULAY_MAX + order[q]] = out[2 + q];
          A[order[q] * PULAY_MAX + slot] = out[2 + q];
        }
        order.push_back(slot);
        PulayMix<T> pm{};
        pm.m = (int)order.size();
        std::vector<double> a, b;
        if (mixer == 1) {
          a = pulay_coefficients(A, order);
          for (double x : a) b.push_back(mix * x);
        } else {
          broyden_coefficients(A, order, mix, a, b);
        }
        for (int q = 0; q < pm.m; ++q) {
          pm.n[q] = hist_n_[order[q]];
          pm.r[q] = hist_r_[order[q]];
          pm.a[q] = a[q];
          pm.b[q] = b[q];
        }
        pulay_mix<T>(nin_, N3, pm, s);
      }
      if (eig_out) std::memcpy(eig_out + (size_t)it * ns_, eig.data(), ns_ * sizeof(double));
      if (resid_out) resid_out[it] = r;
      if (!std::isfinite(r)) fail(KS_ERR_DIVERGED, "scf iteration %d: density residual %g", it, r);
      if (r < tol) {
        ++it;
        break;
      }
    }
    if (iters_done) *iters_done = it;
  }

  // alpha minimising |sum_i alpha_i R_i|^2 with sum_i alpha_i = 1 over the slots in `order`:
  // the bordered system [A 1; 1^T 0] [alpha; mu] = [0; 1], A regularised by 1e-12 of its mean
  // diagonal, solved by Gaussian elimination with partial pivoting (m <= 8).
  static std::vector<double> pulay_coefficients(const std::vector<double>& A, const std::vector<int>& order) {
    const int m = (int)order.size();
    double tr = 0.0;
    for (int i = 0; i < m; ++i) tr += A[order[i] * PULAY_MAX + order[i]];
    const double reg = 1e-12 * std::max(tr / m, 1e-300);
    const int n = m + 1;
    std::vector<double> B((size_t)n * (n + 1), 0.0);
    for (int i = 0; i < m; ++i) {
      for (int j = 0; j < m; ++j) B[i * (n + 1) + j] = A[order[i] * PULAY_MAX + order[j]] + (i == j ? reg : 0.0);
      B[i * (n + 1) + m] = 1.0;
      B[m * (n + 1) + i] = 1.0;
    }
    B[m * (n + 1) + n] = 1.0;                                         // right-hand side (0, ..., 0, 1)
    for (int c = 0; c < n; ++c) {
      int piv = c;
      for (int i = c + 1; i < n; ++i)
        if (std::fabs(B[i * (n + 1) + c]) > std::fabs(B[piv * (n + 1) + c])) piv = i;
      if (piv != c)
        for (int j = 0; j <= n; ++j) std::swap(B[c * (n + 1) + j], B[piv * (n + 1) + j]);
      const double d = B[c * (n + 1) + c];
      if (d == 0.0) fail(KS_ERR_DIVERGED, "scf: singular Pulay system");
      for (int i = 0; i < n; ++i) {
        if (i == c) continue;
        const double f = B[i * (n + 1) + c] / d;
        for (int j = c; j <= n; ++j) B[i * (n + 1) + j] -= f * B[c * (n + 1) + j];
      }
    }
    std::vector<double> alpha(m);
    for (int i = 0; i < m; ++i) alpha[i] = B[i * (n + 1) + n] / B[i * (n + 1) + i];
    return alpha;
  }

  // Broyden's second method (Broyden 1965: the update of the approximate inverse Jacobian)
  // over the window of pairs (x_i, F_i) = (n_in_i, R_i) in `order`, oldest first:
  //   G_0 = -beta I,  G_{j+1} = G_j + u_j dF_j^T / <dF_j|dF_j>,  u_j = dx_j - G_j dF_j,
  //   dx_j = x_{j+1} - x_j, dF_j = F_{j+1} - F_j, and x_next = x_last - G F_last.
  // Every vector involved is a combination of the window's x_i and F_i, so each is carried as
  // its coefficients (over x, over F), and every inner product needed is one of F-combinations,
  // read from the Gram matrix A of the residuals.  Out: x_next = sum_q a_q x_q + b_q F_q.  A
  // pair with <dF_j|dF_j> = 0 carries no update.
  static void broyden_coefficients(const std::vector<double>& A, const std::vector<int>& order, double beta,
                                   std::vector<double>& a, std::vector<double>& b) {
    const int m = (int)order.size();
    auto dot = [&](const std::vector<double>& c1, const std::vector<double>& c2) {   // <sum c1 F|sum c2 F>
      double acc = 0.0;
      for (int i = 0; i < m; ++i)
        for (int k = 0; k < m; ++k) acc += c1[i] * A[order[i] * PULAY_MAX + order[k]] * c2[k];
      return acc;
    };
    auto diff = [&](int j) {                                          // e_{j+1} - e_j
      std::vector<double> e(m, 0.0);
      e[j + 1] = 1.0;
      e[j] = -1.0;
      return e;
    };
    std::vector<std::vector<double>> ux, uF;
    std::vector<double> dd;
    for (int j = 0; j + 1 < m; ++j) {
      const std::vector<double> df = diff(j);
      std::vector<double> gx(m, 0.0), gF(m, 0.0);                     // G_j dF_j
      for (int k = 0; k < m; ++k) gF[k] = -beta * df[k];
      for (int i = 0; i < j; ++i) {
        if (!(dd[i] > 0.0)) continue;
        const double c = dot(diff(i), df) / dd[i];
        for (int k = 0; k < m; ++k) {
          gx[k] += c * ux[i][k];
          gF[k] += c * uF[i][k];
        }
      }
      std::vector<double> uxj(m), uFj(m);
      for (int k = 0; k < m; ++k) {
        uxj[k] = df[k] - gx[k];                                       // dx_j has the coefficients of dF_j
        uFj[k] = -gF[k];
      }
      ux.push_back(uxj);
      uF.push_back(uFj);
      dd.push_back(dot(df, df));
    }
    a.assign(m, 0.0);
    b.assign(m, 0.0);
    a[m - 1] = 1.0;
    b[m - 1] = beta;
    std::vector<double> last(m, 0.0);
    last[m - 1] = 1.0;
    for (int i = 0; i + 1 < m; ++i) {
      if (!(dd[i] > 0.0)) continue;
      const double c = dot(diff(i), last) / dd[i];
      for (int k = 0; k < m; ++k) {
        a[k] -= c * ux[i][k];
        b[k] -= c * uF[i][k];
      }
    }
  }

  // ------------------------------------------------------------------------------------------
  // Delta kick and dipole (Sec. Validation with other codes: a time-localised field at t = 0
  // and the first moment of the density as the observable)
  // ------------------------------------------------------------------------------------------
  // psi_k <- P_S exp(i kappa . (r - L/2)) psi_k, one state at a time through the full-grid
  // work buffer (a once-per-run operation)
  void kick(const double kappa[3], cudaStream_t s) override {
    hpsi_valid_ = false;
    const int N = g_.N;
    const size_t N3 = (size_t)N * N * N;
    ProfScope p(prof, "kick", s);
    for (int b = 0; b < ns_; ++b) {
      C* st = psi_ + (size_t)b * g_.nG;
      KS_CUDA(cudaMemsetAsync(pwork_, 0, N3 * sizeof(C), s));
      scatter_sphere<T>(st, pwork_, t_, 1, s);
      for (int ax = 2; ax >= 0; --ax) fft_axis<T>(pwork_, 1, N, ax, +1, t_.tw, s);
      multiply_phase<T>(pwork_, N, g_.L, kappa, s);
      for (int ax = 0; ax < 3; ++ax) fft_axis<T>(pwork_, 1, N, ax, -1, t_.tw, s);
      gather_kinetic<T>(pwork_, nullptr, st, t_, 1, T(1.0 / double(N3)), s);
    }
  }

  // d = dV sum_j (r_j - L/2) n(r_j) of the resident states' density
  void dipole(double* d_host, cudaStream_t s) override {
    density_of(psi_, ns_, dens_, s);
    ks::dipole<T>(dens_, g_.N, g_.L, dip_partials_, HXC_BLOCKS, dipoles_dev_, s);
    KS_CUDA(cudaMemcpyAsync(d_host, dipoles_dev_, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    KS_CUDA(cudaStreamSynchronize(s));
  }

  // ------------------------------------------------------------------------------------------
  // Forces from the orbital gradients (Eq. 11, with the sign of -dE/dR_I), one state at a time
  // through two full-grid buffers: psi(r) and d_alpha psi(r) from i G_alpha c.
  //   local:    F_Ia -= dV sum_j v_I(r_j) g_a(r_j),  g_a = sum_k f_k 2 Re(conj(d_a psi_k) psi_k)
  //   nonlocal: F_Ia -= sum_k f_k sum_l 2 D Re(conj(q_Il,a) p_Il)
  // v_I is the atom's 27-image Gaussian, separable per axis.
  // ------------------------------------------------------------------------------------------
  void forces(double* f_host, cudaStream_t s) override {
    const int N = g_.N, na = g_.natoms, np = g_.nproj;
    if (na == 0) return;
    const size_t N3 = (size_t)N * N * N;
    force_buffers();
    ProfScope p(prof, "forces", s);
    KS_CUDA(cudaMemsetAsync(fg_, 0, 3 * N3 * sizeof(T), s));
    KS_CUDA(cudaMemsetAsync(fnl_, 0, 3 * (size_t)na * sizeof(double), s));
    const T pscale = T(g_.dV / std::sqrt(g_.omega));   // grids hold Omega^{1/2} psi
    // chunks of fb_ states: psi and one gradient component of every state of the chunk on the
    // full grid, transformed together.  The mixed path transforms with its pruned z-columns
    // and in-SMEM plane passes (planes stored [z][x][y]); the FP64 path with full-grid FFTs.
    bool zmajor = false;
    C* gpack = spare(psi_, hpsi_);                                    // i G_a c of a chunk (packed)
    for (int b0 = 0; b0 < ns_; b0 += fb_) {
      const int nb = std::min(fb_, ns_ - b0);
      const C* st = psi_ + (size_t)b0 * g_.nG;
      auto to_grid = [&](const C* packed, C* grid, int a) {
        if constexpr (sizeof(T) == 4) {
          if (fused_) {
            if (a >= 0) grad_packed<T>(packed, gpack, t_, a, nb, s);
            fused_->real_space(a >= 0 ? gpack : packed, nb, grid, s);
            zmajor = true;
            return;
          }
        }
        KS_CUDA(cudaMemsetAsync(grid, 0, nb * N3 * sizeof(C), s));
        if (a >= 0)
          scatter_grad<T>(packed, grid, t_, a, nb, s);
        else
          scatter_sphere<T>(packed, grid, t_, nb, s);
        for (int ax = 2; ax >= 0; --ax) fft_axis<T>(grid, nb, N, ax, +1, t_.tw, s);
      };
      to_grid(st, fpsi_, -1);
      nl_project<T>(fpsi_, t_, fp_, nb, pscale, s, zmajor);
      for (int a = 0; a < 3; ++a) {
        to_grid(st, fw_, a);
        nl_project<T>(fw_, t_, fq_, nb, pscale, s, zmajor);
        grad_accumulate<T>(fw_, fpsi_, fg_ + a * N3, (int)N3, nb, occ_ + b0, s);
        nl_force<T>(fp_, fq_, na, np, nb, 2.0 * g_.D, occ_ + b0, fnl_, a, s);
      }
    }
    local_force<T>(fg_, fxyz_, N, na, -g_.dV * g_.vloc_depth / g_.omega, flocp_, floc_, s, zmajor);
    std::vector<double> fl(3 * (size_t)na), fn(3 * (size_t)na);
    KS_CUDA(cudaMemcpyAsync(fl.data(), floc_, fl.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    KS_CUDA(cudaMemcpyAsync(fn.data(), fnl_, fn.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    KS_CUDA(cudaStreamSynchronize(s));
    for (size_t i = 0; i < fl.size(); ++i) f_host[i] = fl[i] + fn[i];
  }

  // ------------------------------------------------------------------------------------------
  // Real-time steps: ETRS + Taylor 4 with shared powers (Eqs. 6-8), or plain Taylor 4.
  // ------------------------------------------------------------------------------------------
  void td_steps(double dt, int nsteps, int propagator, int hartree_xc, double* norm_out, double* energy_out,
                double* dipole_out, cudaStream_t s) override {
    hpsi_valid_ = false;
    if (nsteps < 0 || (propagator != 0 && propagator != 1)) fail(KS_ERR_ARG, "td: nsteps=%d propagator=%d", nsteps, propagator);
    if (!hartree_xc) KS_CUDA(cudaMemcpyAsync(vtot_, vloc_, (size_t)g_.N * g_.N * g_.N * sizeof(T), cudaMemcpyDeviceToDevice, s));
    double first_norm = 0;
    bool have_first = false;
    for (int c0 = 0; c0 < nsteps; c0 += MAX_STEPS_CHUNK) {
      const int cn = std::min(MAX_STEPS_CHUNK, nsteps - c0);
      for (int st = 0; st < cn; ++st) td_step_body(dt, propagator, hartree_xc, st, dipole_out != nullptr, nullptr, s);
      std::vector<double> nh(cn), eh(cn), dh(dipole_out ? 3 * cn : 0);
      KS_CUDA(cudaMemcpyAsync(nh.data(), norms_dev_, cn * sizeof(double), cudaMemcpyDeviceToHost, s));
      KS_CUDA(cudaMemcpyAsync(eh.data(), energies_dev_, cn * sizeof(double), cudaMemcpyDeviceToHost, s));
      if (dipole_out)
        KS_CUDA(cudaMemcpyAsync(dh.data(), dipoles_dev_, 3 * cn * sizeof(double), cudaMemcpyDeviceToHost, s));
      KS_CUDA(cudaStreamSynchronize(s));
      check_tc_status(s);
      if (norm_out) std::memcpy(norm_out + c0, nh.data(), cn * sizeof(double));
      if (energy_out) std::memcpy(energy_out + c0, eh.data(), cn * sizeof(double));
      if (dipole_out) std::memcpy(dipole_out + 3 * (size_t)c0, dh.data(), 3 * cn * sizeof(double));
      for (int i = 0; i < cn; ++i) {
        if (!have_first) {
          first_norm = nh[i];
          have_first = true;
        }
        if (!std::isfinite(nh[i]) || !std::isfinite(eh[i]) || std::fabs(nh[i] / first_norm - 1.0) > 0.05)
          fail(KS_ERR_DIVERGED, "real-time step %d: norm %g vs initial %g", c0 + i, nh[i], first_norm);
      }
    }
    // H psi buffer role: keep hpsi_ distinct from psi_
    if (hpsi_ == psi_) hpsi_ = spare(psi_, nullptr);
  }

  // ------------------------------------------------------------------------------------------
  // Moving atoms: the ionic potential and the projectors at new positions, and Ehrenfest
  // dynamics (Sec. "Real-time propagation": velocity-Verlet ions under the forces of Eq. 11,
  // with H(t+dt) of the ETRS step taken at the ions' positions at t + dt).
  // ------------------------------------------------------------------------------------------
  void set_positions(const double* pos, cudaStream_t s) override {
    const int na = g_.natoms;
    if (na == 0) return;
    for (int i = 0; i < 3 * na; ++i)
      if (!std::isfinite(pos[i])) fail(KS_ERR_ARG, "set_positions: position %d is not finite", i);
    // the host lists first: they touch no device memory, so they overlap the kernels still in
    // flight (in Ehrenfest dynamics, the first half of the real-time step)
    build_atoms(pos, g_);
    if constexpr (sizeof(T) == 4) {
      if (fused_) fused_->prepare_atoms();
    }
    // the old lists are released below: wait for this engine's streams (not the whole device, whose
    // other engines keep running)
    KS_CUDA(cudaStreamSynchronize(s));
    KS_CUDA(cudaStreamSynchronize(aux_));
    ProfScope p(prof, "set_positions", s);
    // projector sphere lists (their sizes change as grid points enter and leave the spheres)
    for (const void* q : {(const void*)t_.sph_off, (const void*)t_.sph_idx, (const void*)t_.sph_atom,
                          (const void*)t_.sph_beta, (const void*)t_.sph_zorder, (const void*)t_.cov_idx,
                          (const void*)t_.cov_off, (const void*)t_.cov_ent})
      arena_.release(q);
    t_.sph_off = upload(g_.sph_off);
    t_.sph_idx = upload(g_.sph_idx);
    t_.sph_atom = upload(g_.sph_atom);
    t_.sph_beta = upload_real(g_.sph_beta);
    t_.sph_zorder = upload(g_.sph_zorder);
    t_.cov_idx = upload(g_.cov_idx);
    t_.cov_off = upload(g_.cov_off);
    t_.cov_ent = upload(g_.cov_ent);
    t_.ncov = (int)g_.cov_idx.size();
    KS_CUDA(cudaStreamSynchronize(setup_));                           // the new lists have landed
    update_vloc(s);
    if constexpr (sizeof(T) == 4) {
      if (fused_) fused_->set_atoms(t_);
    }
    hpsi_valid_ = false;
  }

  void ehrenfest(double dt, int nsteps, int hartree_xc, const double* mass, double* vel, double* pos_out,
                 double* energy_out, cudaStream_t s) override {
    const int na = g_.natoms;
    if (nsteps < 0 || !(dt > 0.0) || !std::isfinite(dt)) fail(KS_ERR_ARG, "ehrenfest: nsteps=%d dt=%g", nsteps, dt);
    for (int I = 0; I < na; ++I)
      if (!(mass[I] > 0.0) || !std::isfinite(mass[I])) fail(KS_ERR_ARG, "ehrenfest: mass[%d] = %g", I, mass[I]);
    for (int i = 0; i < 3 * na; ++i)
      if (!std::isfinite(vel[i])) fail(KS_ERR_ARG, "ehrenfest: velocity %d is not finite", i);
    hpsi_valid_ = false;
    const size_t N3 = (size_t)g_.N * g_.N * g_.N;
    if (!hartree_xc) KS_CUDA(cudaMemcpyAsync(vtot_, vloc_, N3 * sizeof(T), cudaMemcpyDeviceToDevice, s));
    std::vector<double> F(3 * (size_t)na), F1(3 * (size_t)na), R1(3 * (size_t)na);
    if (na) forces(F.data(), s);
    double first_norm = 0.0;
    for (int st = 0; st < nsteps; ++st) {
      double kin = 0.0;
      for (int i = 0; i < 3 * na; ++i) {
        const double M = mass[i / 3];
        kin += 0.5 * M * vel[i] * vel[i];
        R1[i] = g_.pos[i] + vel[i] * dt + F[i] * dt * dt / (2.0 * M);
      }
      const std::function<void()> move = [&]() { set_positions(R1.data(), s); };
      td_step_body(dt, 0, hartree_xc, 0, false, na ? &move : nullptr, s);
      double nrm = 0.0, e = 0.0;
      KS_CUDA(cudaMemcpyAsync(&nrm, norms_dev_, sizeof(double), cudaMemcpyDeviceToHost, s));
      KS_CUDA(cudaMemcpyAsync(&e, energies_dev_, sizeof(double), cudaMemcpyDeviceToHost, s));
      KS_CUDA(cudaStreamSynchronize(s));
      check_tc_status(s);
      if (st == 0) first_norm = nrm;
      if (!std::isfinite(nrm) || !std::isfinite(e) || std::fabs(nrm / first_norm - 1.0) > 0.05)
        fail(KS_ERR_DIVERGED, "Ehrenfest step %d: norm %g vs initial %g", st, nrm, first_norm);
      if (na) forces(F1.data(), s);
      for (int i = 0; i < 3 * na; ++i) {
        vel[i] += (F[i] + F1[i]) * dt / (2.0 * mass[i / 3]);
        F[i] = F1[i];
      }
      if (pos_out) std::memcpy(pos_out + 3 * (size_t)na * st, g_.pos.data(), 3 * (size_t)na * sizeof(double));
      if (energy_out) energy_out[st] = e + kin;
    }
    if (hpsi_ == psi_) hpsi_ = spare(psi_, nullptr);
  }

 private:
  // One real-time step from t to t + dt (ETRS with shared powers, or plain Taylor 4) of the
  // resident states of several engines of one precision in lockstep.  norms_dev_[slot] and
  // energies_dev_[slot] of each engine receive its norm and energy at t, dipoles_dev_[3 slot] the
  // dipole when `dipole`; `mid` (one engine only; may be null) runs after the first half and
  // before H(t+dt) is formed (the ions move there).  Every H application of the step runs as one
  // packed launch over the engines where the fused path allows it (fused_apply_h_group), so an
  // engine's results are the same alone and in a group; otherwise engine by engine.
 public:
  static void td_step_group(const std::vector<Engine*>& es, double dt, int propagator, int hartree_xc, int slot,
                            bool dipole, const std::function<void()>* mid, cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value) {
      bool fused = true;
      for (Engine* e : es) fused = fused && e->fused_ != nullptr;
      if (fused) {
        td_step_group_powers(es, dt, propagator, hartree_xc, slot, dipole, mid, s);
        return;
      }
    }
    const size_t ne = es.size();
    std::vector<C*> wa(ne), wb(ne), acc_full(ne), acc_half(ne), wn(ne);
    std::vector<const C*> w(ne), base(ne);
    for (size_t i = 0; i < ne; ++i) {
      Engine* e = es[i];
      const int n = e->ns_, nG = e->g_.nG;
      // roles: psi, two power buffers, acc_full, acc_half
      C* others[5];
      int k = 0;
      for (int q = 0; q < 6; ++q)
        if (e->buf_[q] != e->psi_) others[k++] = e->buf_[q];
      wa[i] = others[0];
      wb[i] = others[1];
      acc_full[i] = others[2];
      acc_half[i] = others[3];
      if (hartree_xc || dipole) e->density_of(e->psi_, n, e->dens_, s);
      if (dipole) ks::dipole<T>(e->dens_, e->g_.N, e->g_.L, e->dip_partials_, HXC_BLOCKS, e->dipoles_dev_ + 3 * slot, s);
      if (hartree_xc) e->update_potential(e->dens_, s);
      state_dots<T>(e->psi_, e->psi_, nG, n, e->dots_, s);
      weighted_energy(e->dots_, e->occ_, n, nullptr, e->norms_dev_ + slot, s);
      w[i] = e->psi_;                 // the accumulators start from psi in the first power's update
    }
    double2 af = make_double2(1, 0), ah = make_double2(1, 0);
    for (int kk = 1; kk <= 4; ++kk) {
      af = cmul_scalar(af, make_double2(0, -dt / kk));
      ah = cmul_scalar(ah, make_double2(0, -0.5 * dt / kk));
      for (size_t i = 0; i < ne; ++i) {
        wn[i] = (w[i] == wa[i]) ? wb[i] : wa[i];
        base[i] = kk == 1 ? es[i]->psi_ : nullptr;
      }
      // H w and both accumulators in one pass; the last power is not stored (nothing reads it)
      group_h(es, w, wn, acc_full, af, propagator == 0 ? acc_half : std::vector<C*>(ne, nullptr), ah, base, kk == 4,
              s);
      for (size_t i = 0; i < ne; ++i) {
        Engine* e = es[i];
        if (kk == 1) {
          state_dots<T>(e->psi_, wn[i], e->g_.nG, e->ns_, e->dots_, s);
          weighted_energy(e->dots_, e->occ_, e->ns_, hartree_xc ? e->parts_ : nullptr, e->energies_dev_ + slot, s);
        }
        w[i] = wn[i];
      }
    }
    if (propagator == 1) {
      for (size_t i = 0; i < ne; ++i) es[i]->psi_ = acc_full[i];
      return;
    }
    if (mid) (*mid)();
    for (size_t i = 0; i < ne; ++i) {
      Engine* e = es[i];
      if (hartree_xc) {
        e->density_of(acc_full[i], e->ns_, e->dens_, s);
        e->update_potential(e->dens_, s);
      }
      w[i] = acc_half[i];
    }
    // second half: out = acc_half + sum_k (-i dt/2)^k/k! H(t+dt)^k acc_half
    ah = make_double2(1, 0);
    for (int kk = 1; kk <= 4; ++kk) {
      ah = cmul_scalar(ah, make_double2(0, -0.5 * dt / kk));
      for (size_t i = 0; i < ne; ++i) {
        wn[i] = (w[i] == wa[i]) ? wb[i] : wa[i];
        base[i] = kk == 1 ? acc_half[i] : nullptr;
      }
      group_h(es, w, wn, acc_full, ah, std::vector<C*>(ne, nullptr), ah, base, kk == 4, s);
      for (size_t i = 0; i < ne; ++i) w[i] = wn[i];
    }
    for (size_t i = 0; i < ne; ++i) es[i]->psi_ = acc_full[i];
  }

 private:
  // td_step_group on the fused path: the first three powers of each Taylor series are kept in
  // three buffers, and the fourth power's epilogue forms the accumulators from them at once
  // (TaylorEpi power-sum form), so the accumulators are written once per series instead of read
  // and written at every power: 15 state-array passes per ETRS step instead of 27, with the same
  // FP32 operations in the same order.
  static void td_step_group_powers(const std::vector<Engine*>& es, double dt, int propagator, int hartree_xc,
                                   int slot, bool dipole, const std::function<void()>* mid, cudaStream_t s) {
    const size_t ne = es.size();
    std::vector<C*> p1(ne), p2(ne), p3(ne), acc_full(ne), acc_half(ne);
    for (size_t i = 0; i < ne; ++i) {
      Engine* e = es[i];
      const int n = e->ns_, nG = e->g_.nG;
      // roles: psi, three powers, acc_full, acc_half
      C* others[5];
      int k = 0;
      for (int q = 0; q < 6; ++q)
        if (e->buf_[q] != e->psi_) others[k++] = e->buf_[q];
      p1[i] = others[0];
      p2[i] = others[1];
      p3[i] = others[2];
      acc_full[i] = others[3];
      acc_half[i] = others[4];
      if (hartree_xc || dipole) e->density_of(e->psi_, n, e->dens_, s);
      if (dipole) ks::dipole<T>(e->dens_, e->g_.N, e->g_.L, e->dip_partials_, HXC_BLOCKS, e->dipoles_dev_ + 3 * slot, s);
      if (hartree_xc) e->update_potential(e->dens_, s);
      state_dots<T>(e->psi_, e->psi_, nG, n, e->dots_, s);
      weighted_energy(e->dots_, e->occ_, n, nullptr, e->norms_dev_ + slot, s);
    }
    // coefficients (-i dt)^k / k! and (-i dt / 2)^k / k!, k = 1..4, formed in FP64 as a running
    // product and rounded to FP32 each
    float2 cf[4], ch[4];
    {
      double2 af = make_double2(1, 0), ah = make_double2(1, 0);
      for (int kk = 1; kk <= 4; ++kk) {
        af = cmul_scalar(af, make_double2(0, -dt / kk));
        ah = cmul_scalar(ah, make_double2(0, -0.5 * dt / kk));
        cf[kk - 1] = make_float2((float)af.x, (float)af.y);
        ch[kk - 1] = make_float2((float)ah.x, (float)ah.y);
      }
    }
    // one Taylor-4 series from the blocks x_i: powers into p1, p2, p3, then out1 (and out2 when
    // set) = x + sum_k c_k H^k x in the fourth power's epilogue
    auto series = [&](const std::vector<const C*>& x, const std::vector<C*>& out1, const float2* c1,
                      const std::vector<C*>* out2, const float2* c2, bool energies, bool cols_ready) {
      std::vector<FusedGroupItem> items(ne);
      const std::vector<C*>* outs[3] = {&p1, &p2, &p3};
      for (int kk = 1; kk <= 4; ++kk) {
        for (size_t i = 0; i < ne; ++i) {
          FusedGroupItem& it = items[i];
          it = FusedGroupItem{};
          it.ops = es[i]->fused_.get();
          it.psi = kk == 1 ? x[i] : (*outs[kk - 2])[i];
          it.n = es[i]->ns_;
          it.cols_ready = kk == 1 && cols_ready;
          it.v = es[i]->vtot_;
          if (kk < 4) {
            it.hpsi = (*outs[kk - 1])[i];
          } else {
            it.hpsi = nullptr;                 // the fourth power is not stored (skip_h)
            it.te.skip_h = 1;
            it.te.nsum = 4;
            it.te.base = x[i];
            it.te.w1 = p1[i];
            it.te.w2 = p2[i];
            it.te.acc1 = out1[i];
            it.te.acc2 = out2 ? (*out2)[i] : nullptr;
            for (int k = 0; k < 4; ++k) {
              it.te.c1[k] = c1[k];
              it.te.c2[k] = c2 ? c2[k] : make_float2(0.f, 0.f);
            }
          }
        }
        {
          ProfScope scope(es[0]->prof, "apply_h", s);
          fused_apply_h_group(items, s);
        }
        if (energies && kk == 1)
          for (size_t i = 0; i < ne; ++i) {
            Engine* e = es[i];
            state_dots<T>(e->psi_, p1[i], e->g_.nG, e->ns_, e->dots_, s);
            weighted_energy(e->dots_, e->occ_, e->ns_, hartree_xc ? e->parts_ : nullptr, e->energies_dev_ + slot,
                            s);
          }
      }
    };
    std::vector<const C*> x(ne);
    for (size_t i = 0; i < ne; ++i) x[i] = es[i]->psi_;
    // the density of psi just ran on the fused path and left the z transform of psi in each
    // cell's column buffer: the first H application of psi starts from it
    series(x, acc_full, cf, propagator == 0 ? &acc_half : nullptr, ch, true, hartree_xc || dipole);
    if (propagator == 1) {
      for (size_t i = 0; i < ne; ++i) es[i]->psi_ = acc_full[i];
      return;
    }
    if (mid) (*mid)();
    for (size_t i = 0; i < ne; ++i) {
      Engine* e = es[i];
      if (hartree_xc) {
        e->density_of(acc_full[i], e->ns_, e->dens_, s);
        e->update_potential(e->dens_, s);
      }
      x[i] = acc_half[i];
    }
    // second half: psi(t + dt) = acc_half + sum_k (-i dt/2)^k/k! H(t+dt)^k acc_half
    series(x, acc_full, ch, nullptr, nullptr, false, false);
    for (size_t i = 0; i < ne; ++i) es[i]->psi_ = acc_full[i];
  }

  // wn_i = H w_i for every engine, with acc1_i <- base_i + a1 wn_i and acc2_i <- base_i + a2 wn_i
  // (base null: each accumulator's own value): one packed fused launch per kernel when every
  // engine has the fused path, else engine by engine (H application, then one accumulation pass).
  static void group_h(const std::vector<Engine*>& es, const std::vector<const C*>& w, const std::vector<C*>& wn,
                      const std::vector<C*>& acc1, double2 a1, const std::vector<C*>& acc2, double2 a2,
                      const std::vector<const C*>& base, bool skip_h, cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value) {
      bool fused = true;
      for (Engine* e : es) fused = fused && e->fused_ != nullptr;
      if (fused) {
        ProfScope scope(es[0]->prof, "apply_h", s);
        std::vector<FusedGroupItem> items(es.size());
        for (size_t i = 0; i < es.size(); ++i) {
          FusedGroupItem& it = items[i];
          it.ops = es[i]->fused_.get();
          it.psi = w[i];
          it.hpsi = wn[i];
          it.n = es[i]->ns_;
          it.v = es[i]->vtot_;
          it.te.acc1 = acc1[i];
          it.te.a1 = make_float2((float)a1.x, (float)a1.y);
          it.te.acc2 = acc2[i];
          it.te.a2 = make_float2((float)a2.x, (float)a2.y);
          it.te.base = base[i];
          it.te.base_is_psi = base[i] != nullptr && base[i] == w[i];
          it.te.skip_h = skip_h ? 1 : 0;
        }
        fused_apply_h_group(items, s);
        return;
      }
    }
    for (size_t i = 0; i < es.size(); ++i) {
      Engine* e = es[i];
      e->apply_h(w[i], wn[i], e->ns_, s);
      axpy2<T>(acc1[i], a1, acc2[i], a2, wn[i], base[i], (size_t)e->ns_ * e->g_.nG, s);
    }
  }

  void td_step_body(double dt, int propagator, int hartree_xc, int slot, bool dipole, const std::function<void()>* mid,
                    cudaStream_t s) {
    td_step_group(std::vector<Engine*>{this}, dt, propagator, hartree_xc, slot, dipole, mid, s);
  }

  // V = V_loc from the separable 27-image Gaussians of the current positions, in FP64 on the
  // device, kept in FP64 (vloc64_) beside the working precision, with its extremes on the host
  // (the steepest-descent step uses them).
  void update_vloc(cudaStream_t s) {
    const int N = g_.N;
    const size_t N3 = (size_t)N * N * N;
    build_axis_tables(s);
    vloc_from_axes<T>(fxyz_, g_.natoms, N, g_.vloc_depth, vloc_, vloc64_, s);
    KS_CUDA(cudaMemcpyAsync(vtot_, vloc_, N3 * sizeof(T), cudaMemcpyDeviceToDevice, s));
    minmax(vloc64_, N3, hxc_partials_, HXC_BLOCKS, vmm_, s);
    double mm[2];
    KS_CUDA(cudaMemcpyAsync(mm, vmm_, sizeof(mm), cudaMemcpyDeviceToHost, s));
    KS_CUDA(cudaStreamSynchronize(s));
    g_.vmin = mm[0];
    g_.vmax = mm[1];
  }

  void get_vloc(double* v_host) override {
    KS_CUDA(cudaMemcpy(v_host, vloc64_, (size_t)g_.N * g_.N * g_.N * sizeof(double), cudaMemcpyDeviceToHost));
  }

  // Work buffers of the force evaluation (allocated on first use): full grids for a chunk of
  // fb_ states (at most 2 GB for the two), their projections, the gradient densities.
  void force_buffers() {
    if (fw_) return;
    const int N = g_.N, na = g_.natoms, np = g_.nproj;
    const size_t N3 = (size_t)N * N * N;
    fb_ = (int)std::max<size_t>(1, std::min<size_t>((size_t)ns_, (size_t(2048) << 20) / (2 * N3 * sizeof(C))));
    fpsi_ = alloc<C>((size_t)fb_ * N3);
    fw_ = alloc<C>((size_t)fb_ * N3);
    fg_ = alloc<T>(3 * N3);
    fp_ = alloc<C>((size_t)fb_ * na * np);
    fq_ = alloc<C>((size_t)fb_ * na * np);
    fnl_ = alloc<double>(3 * (size_t)na);
    floc_ = alloc<double>(3 * (size_t)na);
    flocp_ = alloc<double>(3 * (size_t)na * LOCAL_FORCE_SPLIT);
  }

  // Per atom and axis: X_a(x) = sum_{s = -1, 0, 1} exp(-(x - R_a - L s)^2 / (2 w^2)) on the
  // grid; V_loc = A sum_a X_a(x) Y_a(y) Z_a(z) and the local force both use them.
  void build_axis_tables(cudaStream_t s) {
    const int N = g_.N, na = g_.natoms;
    if (!fxyz_) fxyz_ = alloc<double>(std::max<size_t>(1, 3 * (size_t)na * N));
    std::vector<double> xyz(3 * (size_t)na * N);
    const double w2 = 2.0 * g_.vloc_width * g_.vloc_width;
    for (int I = 0; I < na; ++I)
      for (int a = 0; a < 3; ++a)
        for (int j = 0; j < N; ++j) {
          double v = 0.0;
          for (int sh = -1; sh <= 1; ++sh) {
            const double dx = g_.h * j - g_.pos[3 * I + a] - g_.L * sh;
            v += std::exp(-dx * dx / w2);
          }
          xyz[((size_t)I * 3 + a) * N + j] = v;
        }
    KS_CUDA(cudaMemcpyAsync(fxyz_, xyz.data(), xyz.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  }
  static double2 cmul_scalar(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
  }

  // A state buffer that is neither a nor b.
  C* spare(const C* a, const C* b) {
    for (int i = 0; i < 6; ++i)
      if (buf_[i] != a && buf_[i] != b) return buf_[i];
    fail(KS_ERR_STATE, "internal: no spare state buffer");
  }
  bool use_tc() const { return sizeof(T) == 4 && prec_ == KS_MIXED_BF16X3; }
  bool mixed_cholesky() const { return sizeof(T) == 4 && ns_ <= 256; }
  // the mixed path's FP32 eigensolver: one-CTA Householder for n <= 128, one-CTA FP32 Jacobi up
  // to 256 (both finished by FP64 Rayleigh quotients); FP64 Jacobi beyond, or with
  // KS_OPT_FP64_SUBSPACE
  void eigh_sub(int n, double2* Vt, cudaStream_t s) {
    if (sizeof(T) == 4 && !fp64_subspace_ && n <= 128)
      eigh_mixed(mA_, mV_, lam_, eig_, Vt, n, s);
    else if (sizeof(T) == 4 && !fp64_subspace_ && n <= 256)
      eigh_jacobi_mixed(mA_, mV_, lam_, eig_, Vt, reinterpret_cast<float2*>(mF_), n, s);
    else
      jacobi_eigh(mA_, mV_, eig_, Vt, n, s);
  }
  // KS_OPT_FP64_SUBSPACE on a mixed handle: the Cholesky factor of S, the subspace products and
  // the Rayleigh-Ritz eigensolver in FP64 (as on the FP64 path), the states and their GEMMs mixed
  bool fp64_subspace_ = false;
  // the block iteration's Rayleigh-Ritz step runs in one CTA (rr_step_mixed)
  bool fused_rr() const { return use_tc() && ns_ <= 128; }

  // out = A^H B over the sphere (n x n), tensor cores on the bf16x3 mixed path
  void overlap(const C* A, const C* B, int n, double2* out, cudaStream_t s, float2* out32 = nullptr) {
    if constexpr (std::is_same<T, float>::value) {
      if (use_tc()) {
        tc_overlap(A, g_.nG, B, g_.nG, n, n, g_.nG, part_, part_elems_, out, status_ + 1, s, out32);
        return;
      }
    }
    gemm_cn<T>(A, g_.nG, B, g_.nG, n, n, g_.nG, part_, part_elems_, out, s);
  }

  // Y = M X (rows of states); with X2, M is n x 2n and X = [X; X2]
  void rot(const double2* M, const C* X, C* Y, cudaStream_t s, const C* X2 = nullptr) {
    const int nin = X2 ? 2 * ns_ : ns_;
    if constexpr (std::is_same<T, float>::value) {
      if (use_tc()) {
        tc_rotate(M, nin, X, X2, ns_, g_.nG, Y, g_.nG, ns_, g_.nG, rotws_, rotws_bytes_, status_ + 1, s);
        return;
      }
    }
    rotate<T>(M, nin, X, X2, ns_, g_.nG, Y, g_.nG, ns_, g_.nG, s);
  }

  // Y = Mcat [X; X2] from the split image of mcat32_ that tc_rotate_prepare left in rotws_
  void rot_prepared(const C* X, const C* X2, C* Y, cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value)
      tc_rotate_prepared(rotws_, 2 * ns_, X, X2, ns_, g_.nG, Y, g_.nG, ns_, g_.nG, status_ + 1, s);
    else
      fail(KS_ERR_STATE, "internal: prepared rotation on the FP64 path");
  }

  void check_tc_status(cudaStream_t s) {
    int e = 0;
    KS_CUDA(cudaMemcpyAsync(&e, status_ + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    KS_CUDA(cudaStreamSynchronize(s));
    if (e) KS_CUDA(cudaMemsetAsync(status_ + 1, 0, sizeof(int), s));
    raise_tc_status(e);
  }

  C* spare3(const C* a, const C* b, const C* c) {
    for (int i = 0; i < 6; ++i)
      if (buf_[i] != a && buf_[i] != b && buf_[i] != c) return buf_[i];
    fail(KS_ERR_STATE, "internal: no spare state buffer");
  }
  C* spare4(const C* a, const C* b, const C* c, const C* d) {
    for (int i = 0; i < 6; ++i)
      if (buf_[i] != a && buf_[i] != b && buf_[i] != c && buf_[i] != d) return buf_[i];
    fail(KS_ERR_STATE, "internal: no spare state buffer");
  }
  void swap_in(C*& role, C* fresh) { role = fresh; }

  template <typename U> U* alloc(size_t n) { return static_cast<U*>(arena_.alloc(n * sizeof(U))); }
  template <typename U> const U* upload(const std::vector<U>& v) {
    U* p = alloc<U>(std::max<size_t>(v.size(), 1));
    if (!v.empty()) KS_CUDA(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(U), cudaMemcpyHostToDevice, setup_));
    return p;
  }
  const T* upload_real(const std::vector<double>& v) {
    std::vector<T> t(v.begin(), v.end());
    return upload(t);
  }

  HostGeometry g_;
  ks_precision prec_;
  int ns_;
  DeviceArena arena_;
  DevTables<T> t_;
  std::unique_ptr<FusedOps> fused_;
  T* vloc_ = nullptr;
  double* vloc64_ = nullptr;        // V_loc in FP64 (the ABI's copy), and its min and max
  double* vmm_ = nullptr;
  T* vtot_ = nullptr;
  double* occ_ = nullptr;
  C* buf_[6] = {};
  C* psi_ = nullptr;
  C* hpsi_ = nullptr;
  double2* staging_ = nullptr;
  C* grid_ = nullptr;
  C* proj_ = nullptr;
  int batch_ = 1;
  double2* part_ = nullptr;
  size_t part_elems_ = 0;
  double2 *mS_ = nullptr, *mA_ = nullptr, *mM_ = nullptr, *mV_ = nullptr;
  double* eig_ = nullptr;
  double* lam_ = nullptr;
  double2* chw_ = nullptr;   // two-pass FP32 Cholesky workspace (mixed path)
  double2 *mT_ = nullptr, *mC_ = nullptr, *mF_ = nullptr;   // subspace products, FP64 factor scratch
  double2* mCat_ = nullptr;                                   // [n][2n] steepest-descent step matrix
  // one-CTA Rayleigh-Ritz step of the block iteration (FP32 operands and results)
  float2 *hraw32_ = nullptr, *m32_ = nullptr, *mcat32_ = nullptr, *aexp_ = nullptr, *vexp_ = nullptr;
  int* perm_ = nullptr;
  cudaStream_t setup_ = nullptr;     // = aux_: setup work at creation and at atom moves
  // hpsi_ = H psi_ for the resident block (kept by the block iteration between calls); after
  // HPSI_REFRESH iterations that derived it by recurrence, H is applied to psi_ afresh.
  static constexpr int HPSI_REFRESH = 16;
  bool hpsi_valid_ = false;
  int hpsi_age_ = 0;
  cudaStream_t aux_ = nullptr;
  cudaEvent_t ev_gram_ = nullptr, ev_hraw_ = nullptr, ev_chol_ = nullptr, ev_ritz_ = nullptr;
  void* rotws_ = nullptr;
  size_t rotws_bytes_ = 0;
  int* status_ = nullptr;
  T* dens_ = nullptr;
  C* pwork_ = nullptr;
  double* hxc_partials_ = nullptr;
  T* nin_ = nullptr;                // SCF input density
  double* resid_dev_ = nullptr;     // SCF residual
  double* dip_partials_ = nullptr;  // dipole block partials
  double2* trr_ = nullptr;          // per-state residual kinetic sums of the preconditioned update
  C* fw_ = nullptr;                 // forces: state and gradient grids of a chunk, accumulators,
  C* fpsi_ = nullptr;               // projections (on first use)
  int fb_ = 1;
  T* fg_ = nullptr;
  C *fp_ = nullptr, *fq_ = nullptr;
  double *fnl_ = nullptr, *floc_ = nullptr, *flocp_ = nullptr, *fxyz_ = nullptr;
  T* hist_n_[PULAY_MAX] = {};       // Pulay history: input densities and residuals (allocated on first use)
  T* hist_r_[PULAY_MAX] = {};
  double* pulay_partials_ = nullptr;
  double* pulay_out_ = nullptr;
  double* dipoles_dev_ = nullptr;   // [MAX_STEPS_CHUNK][3] dipoles of a chunk of real-time steps
  double* parts_ = nullptr;
  double2* dots_ = nullptr;
  double* norms_dev_ = nullptr;
  double* energies_dev_ = nullptr;
};

}  // namespace

void raise_tc_status(int flag) {
  if (flag) fail(KS_ERR_CUDA, "tensor-core GEMM: a bounded wait expired (error flag %d)", flag);
}

bool td_groupable(const EngineBase* a, const EngineBase* b) {
  if (a->precision() != KS_MIXED_BF16X3 || b->precision() != KS_MIXED_BF16X3) return false;
  const auto* ea = dynamic_cast<const Engine<float>*>(a);
  const auto* eb = dynamic_cast<const Engine<float>*>(b);
  return ea && eb && ea->groupable_with(*eb);
}

void td_step_engines(const std::vector<EngineBase*>& es, double dt, int hartree_xc, double* norms, double* energies,
                     cudaStream_t s) {
  if (es.empty()) return;
  std::vector<Engine<float>*> ef;
  for (EngineBase* e : es) {
    auto* p = dynamic_cast<Engine<float>*>(e);
    if (!p || !td_groupable(es[0], e)) fail(KS_ERR_ARG, "td_step_engines: engines that cannot share launches");
    ef.push_back(p);
  }
  for (auto* e : ef) e->td_prepare(hartree_xc, s);
  Engine<float>::td_step_group(ef, dt, 0, hartree_xc, 0, false, nullptr, s);
  for (size_t i = 0; i < ef.size(); ++i) ef[i]->td_read_slot0(norms + i, energies + i, s);
  KS_CUDA(cudaStreamSynchronize(s));
  for (size_t i = 0; i < ef.size(); ++i) {
    ef[i]->td_finish(s);
    if (!std::isfinite(norms[i]) || !std::isfinite(energies[i]))
      fail(KS_ERR_DIVERGED, "real-time step: norm %g, energy %g", norms[i], energies[i]);
  }
}

std::unique_ptr<EngineBase> make_engine(const ks_cell_desc& d, DevicePool* pool) {
  if (d.prec == KS_FP64) return std::unique_ptr<EngineBase>(new Engine<double>(d, pool));
  if (d.prec == KS_MIXED_BF16X3) return std::unique_ptr<EngineBase>(new Engine<float>(d, pool));
  fail(KS_ERR_ARG, "unknown precision %d", (int)d.prec);
}

}  // namespace ks
