// The C ABI (include/ks.h): argument checks, handle lifetime, and translation of internal
// errors into ks_status.  No exception crosses this boundary.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>

#include "engine.h"
#include "tuner.h"

namespace ks {
const char* last_error_cstr();
uint64_t launch_count();
}

struct ks_grid_s {
  std::unique_ptr<ks::EngineBase> eng;
};

namespace {

template <typename F> ks_status guarded(F&& f) {
  try {
    f();
    return KS_OK;
  } catch (const ks::Error& e) {
    return e.st;
  } catch (const std::bad_alloc&) {
    ks::set_last_error("host allocation failed");
    return KS_ERR_NOMEM;
  } catch (...) {
    ks::set_last_error("unexpected internal error");
    return KS_ERR_CUDA;
  }
}

inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

void need(bool ok, const char* what) {
  if (!ok) ks::fail(KS_ERR_ARG, "%s", what);
}

}  // namespace

extern "C" {

const char* ks_last_error(void) { return ks::last_error_cstr(); }

ks_status ks_count_gvectors(double L, int N, double ecut, int* nG) {
  return guarded([&] {
    need(nG != nullptr, "nG is NULL");
    ks::count_sphere(L, N, ecut, nG);
  });
}

ks_status ks_grid_create(const ks_cell_desc* desc, ks_grid* out) {
  if (out) *out = nullptr;
  return guarded([&] {
    need(desc != nullptr && out != nullptr, "desc/out is NULL");
    std::unique_ptr<ks_grid_s> g(new ks_grid_s);
    g->eng = ks::make_engine(*desc);
    *out = g.release();
  });
}

ks_status ks_grid_destroy(ks_grid g) {
  return guarded([&] {
    if (g) {
      cudaDeviceSynchronize();
      delete g;
    }
  });
}

ks_status ks_grid_gvectors(ks_grid g, int* nG, int* m) {
  return guarded([&] {
    need(g && nG, "grid/nG is NULL");
    const auto& geo = g->eng->geo();
    *nG = geo.nG;
    if (m) std::memcpy(m, geo.mvec.data(), geo.mvec.size() * sizeof(int));
  });
}

ks_status ks_grid_device_bytes(ks_grid g, size_t* bytes) {
  return guarded([&] {
    need(g && bytes, "grid/bytes is NULL");
    *bytes = g->eng->device_bytes();
  });
}

ks_status ks_get_vloc(ks_grid g, double* v_host) {
  return guarded([&] {
    need(g && v_host, "grid/v is NULL");
    g->eng->get_vloc(v_host);
  });
}

ks_status ks_set_states(ks_grid g, const double* c_host) {
  return guarded([&] {
    need(g && c_host, "grid/c is NULL");
    g->eng->set_states(c_host, 0);
  });
}

ks_status ks_get_states(ks_grid g, double* c_host) {
  return guarded([&] {
    need(g && c_host, "grid/c is NULL");
    g->eng->get_states(c_host, 0);
  });
}

ks_status ks_states_device(ks_grid g, void** psi_dev) {
  return guarded([&] {
    need(g && psi_dev, "grid/psi_dev is NULL");
    *psi_dev = g->eng->states_device();
  });
}

ks_status ks_apply_h(ks_grid g, const void* psi_dev, void* hpsi_dev, int nstates, void* stream) {
  return guarded([&] {
    need(g && psi_dev && hpsi_dev, "grid/psi/hpsi is NULL");
    need(psi_dev != hpsi_dev, "psi and hpsi must not overlap");
    g->eng->apply_h(psi_dev, hpsi_dev, nstates, as_stream(stream));
  });
}

ks_status ks_apply_h_host(ks_grid g, const double* psi_host, double* hpsi_host, int nstates) {
  return guarded([&] {
    need(g && psi_host && hpsi_host, "grid/psi/hpsi is NULL");
    g->eng->apply_h_host(psi_host, hpsi_host, nstates);
  });
}

ks_status ks_density(ks_grid g, void* n_dev, void* stream) {
  return guarded([&] {
    need(g && n_dev, "grid/n is NULL");
    g->eng->density(n_dev, as_stream(stream));
  });
}

ks_status ks_orthonormalize(ks_grid g, double* S_host_opt, void* stream) {
  return guarded([&] {
    need(g != nullptr, "grid is NULL");
    g->eng->orthonormalize(S_host_opt, as_stream(stream));
  });
}

ks_status ks_rayleigh_ritz(ks_grid g, double* eig_host, void* stream) {
  return guarded([&] {
    need(g != nullptr, "grid is NULL");
    g->eng->rayleigh_ritz(eig_host, as_stream(stream));
  });
}

ks_status ks_block_iteration(ks_grid g, int niter, double* eig_host, void* stream) {
  return guarded([&] {
    need(g != nullptr, "grid is NULL");
    g->eng->block_iteration(niter, eig_host, as_stream(stream));
  });
}

ks_status ks_td_step(ks_grid g, double dt, int nsteps, int propagator, int hartree_xc, double* norm_out,
                     double* energy_out, void* stream) {
  return guarded([&] {
    need(g != nullptr, "grid is NULL");
    need(dt > 0 && dt < 10, "dt must be in (0, 10)");
    g->eng->td_steps(dt, nsteps, propagator, hartree_xc, norm_out, energy_out, nullptr, as_stream(stream));
  });
}

ks_status ks_td_step_dipole(ks_grid g, double dt, int nsteps, int propagator, int hartree_xc, double* norm_out,
                            double* energy_out, double* dipole_out, void* stream) {
  return guarded([&] {
    need(g != nullptr, "grid is NULL");
    need(dt > 0 && dt < 10, "dt must be in (0, 10)");
    g->eng->td_steps(dt, nsteps, propagator, hartree_xc, norm_out, energy_out, dipole_out, as_stream(stream));
  });
}

ks_status ks_kick(ks_grid g, const double* kappa, void* stream) {
  return guarded([&] {
    need(g != nullptr && kappa != nullptr, "grid or kappa is NULL");
    for (int i = 0; i < 3; ++i) need(std::isfinite(kappa[i]), "kappa must be finite");
    g->eng->kick(kappa, as_stream(stream));
  });
}

ks_status ks_forces(ks_grid g, double* f_out, void* stream) {
  return guarded([&] {
    need(g != nullptr && f_out != nullptr, "grid or f_out is NULL");
    g->eng->forces(f_out, as_stream(stream));
  });
}

ks_status ks_set_positions(ks_grid g, const double* pos, void* stream) {
  return guarded([&] {
    need(g != nullptr && (pos != nullptr || g->eng->geo().natoms == 0), "grid or pos is NULL");
    g->eng->set_positions(pos, as_stream(stream));
  });
}

ks_status ks_get_positions(ks_grid g, double* pos) {
  return guarded([&] {
    need(g != nullptr && (pos != nullptr || g->eng->geo().natoms == 0), "grid or pos is NULL");
    const auto& geo = g->eng->geo();
    if (geo.natoms) std::memcpy(pos, geo.pos.data(), 3 * (size_t)geo.natoms * sizeof(double));
  });
}

ks_status ks_ehrenfest(ks_grid g, double dt, int nsteps, int hartree_xc, const double* mass, double* vel,
                       double* pos_out, double* energy_out, void* stream) {
  return guarded([&] {
    need(g != nullptr, "grid is NULL");
    need(g->eng->geo().natoms == 0 || (mass != nullptr && vel != nullptr), "mass or vel is NULL");
    g->eng->ehrenfest(dt, nsteps, hartree_xc, mass, vel, pos_out, energy_out, as_stream(stream));
  });
}

ks_status ks_dipole(ks_grid g, double* d_out, void* stream) {
  return guarded([&] {
    need(g != nullptr && d_out != nullptr, "grid or d_out is NULL");
    g->eng->dipole(d_out, as_stream(stream));
  });
}

ks_status ks_autotune_report(char* buf, size_t cap, size_t* len) {
  return guarded([&] {
    const std::string j = ks::tune_log_json();
    if (len) *len = j.size() + 1;
    if (buf && cap > 0) {
      const size_t k = std::min(cap - 1, j.size());
      std::memcpy(buf, j.data(), k);
      buf[k] = 0;
    }
  });
}

ks_status ks_tc_status_check(int flag) {
  return guarded([&] { ks::raise_tc_status(flag); });
}

ks_status ks_set_option(ks_grid g, int option, int value) {
  return guarded([&] {
    need(g != nullptr, "grid is NULL");
    g->eng->set_option(option, value);
  });
}

ks_status ks_block_iteration_pc(ks_grid g, int niter, int precond, double* eig_host, void* stream) {
  return guarded([&] {
    need(g != nullptr, "grid is NULL");
    need(niter >= 0 && (precond == 0 || precond == 1), "block_iteration_pc: niter >= 0, precond 0 or 1");
    if (precond == 0)
      g->eng->block_iteration(niter, eig_host, as_stream(stream));
    else
      g->eng->block_iteration_teter(niter, eig_host, as_stream(stream));
  });
}

ks_status ks_scf(ks_grid g, int max_iter, int eig_iters, int mixer, double mix, int history, double tol,
                 double* eig_out, double* resid_out, int* iters_done, void* stream) {
  return guarded([&] {
    need(g != nullptr, "grid is NULL");
    need(max_iter >= 0 && eig_iters >= 1 && mixer >= 0 && mixer <= 2 && mix > 0.0 && mix <= 1.0 &&
             history >= 1 && history <= 8 && tol >= 0.0,
         "scf: need max_iter >= 0, eig_iters >= 1, mixer 0, 1 or 2, 0 < mix <= 1, 1 <= history <= 8, tol >= 0");
    g->eng->scf(max_iter, eig_iters, mixer, mix, history, tol, eig_out, resid_out, iters_done, as_stream(stream));
  });
}

ks_status ks_profile(ks_grid g, int mode) {
  return guarded([&] {
    need(g != nullptr && mode >= 0 && mode <= 4, "grid is NULL or mode not in 0..4");
    if (mode == 2)
      g->eng->prof.reset();
    else if (mode >= 3)
      g->eng->prof.timeline(mode == 3);
    else
      g->eng->prof.enable(mode == 1);
  });
}

ks_status ks_profile_read(ks_grid g, int idx, char* name, int name_len, double* ms, long* count) {
  return guarded([&] {
    need(g && name && name_len > 0 && ms && count, "bad profile_read arguments");
    g->eng->prof.collect();
    const auto& e = g->eng->prof.entries();
    if (idx < 0 || idx >= (int)e.size()) ks::fail(KS_ERR_ARG, "profile entry %d of %d", idx, (int)e.size());
    std::snprintf(name, name_len, "%s", e[idx].name.c_str());
    *ms = e[idx].ms;
    *count = e[idx].count;
  });
}

ks_status ks_profile_span(ks_grid g, int idx, char* name, int name_len, double* start_ms, double* end_ms) {
  return guarded([&] {
    need(g && name && name_len > 0 && start_ms && end_ms, "bad profile_span arguments");
    g->eng->prof.collect();
    const auto& sp = g->eng->prof.spans();
    if (idx < 0 || idx >= (int)sp.size()) ks::fail(KS_ERR_ARG, "profile span %d of %d", idx, (int)sp.size());
    std::snprintf(name, name_len, "%s", g->eng->prof.entries()[sp[idx].entry].name.c_str());
    *start_ms = sp[idx].start;
    *end_ms = sp[idx].end;
  });
}

uint64_t ks_kernel_launches(void) { return ks::launch_count(); }

}  // extern "C"
