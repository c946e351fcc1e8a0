// Host-side setup of one cell: the plane-wave cutoff sphere and its z-columns, the local
// potential on the grid, and the real-space projector spheres (Sec. "Pseudopotentials",
// Eq. 9).  Built once per handle in FP64 and copied to the device.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <map>

#include "common.h"

namespace ks {

static thread_local std::string g_last_error = "no error";
static std::atomic<uint64_t> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

void set_last_error(const std::string& msg) { g_last_error = msg; }
const char* last_error_cstr() { return g_last_error.c_str(); }

void fail(ks_status st, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  throw Error{st};
}

void fail_cuda(cudaError_t e, const char* what, const char* file, int line) {
  char buf[1024];
  snprintf(buf, sizeof buf, "CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
  set_last_error(buf);
  throw Error{e == cudaErrorMemoryAllocation ? KS_ERR_NOMEM : KS_ERR_CUDA};
}

bool valid_fft_length(int N) {
  if (N < 8 || N > 128 || (N & 1)) return false;
  int n = N;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

static inline int freq(int j, int N) { return (2 * j < N) ? j : j - N; }

// Squared-radius bound in integer units: (2 pi / L)^2 |m|^2 / 2 <= ecut  <=>  |m|^2 <= B.
static inline double sphere_bound(double L, double ecut) {
  const double s = L / (2.0 * M_PI);
  return 2.0 * ecut * s * s;
}

void count_sphere(double L, int N, double ecut, int* nG) {
  if (!(L > 0) || !(ecut > 0) || !valid_fft_length(N)) fail(KS_ERR_ARG, "bad cell: L=%g N=%d ecut=%g", L, N, ecut);
  const double B = sphere_bound(L, ecut);
  const int mmax = (int)std::floor(std::sqrt(B));
  if (2 * mmax >= N) fail(KS_ERR_ARG, "cutoff sphere (|m| <= %d) does not fit the %d^3 grid", mmax, N);
  long count = 0;
  for (int jx = 0; jx < N; ++jx)
    for (int jy = 0; jy < N; ++jy)
      for (int jz = 0; jz < N; ++jz) {
        const int mx = freq(jx, N), my = freq(jy, N), mz = freq(jz, N);
        const double g2 = (2.0 * M_PI / L) * (2.0 * M_PI / L) * double(mx * mx + my * my + mz * mz);
        if (0.5 * g2 <= ecut) ++count;
      }
  *nG = (int)count;
}

void build_atoms(const double* pos, HostGeometry& g, bool with_vloc) {
  const int N = g.N;
  const double L = g.L;
  // ---- V_loc(r) = sum_a A exp(-|r - R_a - L n|^2 / (2 w^2)) over the 27 image shifts -------
  // Terms with |r - R_a - L n| > 10 w are below 2e-22 |A| and are skipped.
  g.pos.assign(pos ? pos : nullptr, pos ? pos + 3 * (size_t)g.natoms : nullptr);
  const double w2 = 2.0 * g.vloc_width * g.vloc_width;
  const double rcut = 10.0 * g.vloc_width;
  if (with_vloc) g.vloc.assign((size_t)N * N * N, 0.0);
  for (int a = 0; a < g.natoms && with_vloc; ++a) {
    const double R[3] = {pos[3 * a], pos[3 * a + 1], pos[3 * a + 2]};
    for (int sx = -1; sx <= 1; ++sx)
      for (int sy = -1; sy <= 1; ++sy)
        for (int sz = -1; sz <= 1; ++sz) {
          const double C[3] = {R[0] + L * sx, R[1] + L * sy, R[2] + L * sz};
          int lo[3], hi[3];
          for (int k = 0; k < 3; ++k) {
            lo[k] = std::max(0, (int)std::floor((C[k] - rcut) / g.h));
            hi[k] = std::min(N - 1, (int)std::ceil((C[k] + rcut) / g.h));
          }
          for (int jx = lo[0]; jx <= hi[0]; ++jx)
            for (int jy = lo[1]; jy <= hi[1]; ++jy)
              for (int jz = lo[2]; jz <= hi[2]; ++jz) {
                const double dx = jx * g.h - C[0], dy = jy * g.h - C[1], dz = jz * g.h - C[2];
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 > rcut * rcut) continue;
                g.vloc[((size_t)jx * N + jy) * N + jz] += g.vloc_depth * std::exp(-r2 / w2);
              }
        }
  }
  if (with_vloc) {
    g.vmin = *std::min_element(g.vloc.begin(), g.vloc.end());
    g.vmax = *std::max_element(g.vloc.begin(), g.vloc.end());
  }

  // ---- projector spheres |d| < R_c around each atom (minimum image), grid order ----------
  g.sph_off.assign(1, 0);
  g.sph_idx.clear();
  g.sph_atom.clear();
  g.sph_beta.clear();
  const double s2 = 2.0 * g.proj_sigma * g.proj_sigma;
  const double rc2 = g.proj_rc * g.proj_rc;
  for (int a = 0; a < g.natoms; ++a) {
    const double R[3] = {pos[3 * a], pos[3 * a + 1], pos[3 * a + 2]};
    std::vector<int> pts;
    int lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
      lo[k] = (int)std::floor((R[k] - g.proj_rc) / g.h) - 1;
      hi[k] = (int)std::ceil((R[k] + g.proj_rc) / g.h) + 1;
    }
    for (int ix = lo[0]; ix <= hi[0]; ++ix)
      for (int iy = lo[1]; iy <= hi[1]; ++iy)
        for (int iz = lo[2]; iz <= hi[2]; ++iz) {
          const int jx = ((ix % N) + N) % N, jy = ((iy % N) + N) % N, jz = ((iz % N) + N) % N;
          pts.push_back((jx * N + jy) * N + jz);
        }
    std::sort(pts.begin(), pts.end());
    pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
    std::vector<int> inside;
    std::vector<double> dd;
    for (int p : pts) {
      const int jx = p / (N * N), jy = (p / N) % N, jz = p % N;
      const int j3[3] = {jx, jy, jz};
      double dv[3], r2 = 0;
      for (int k = 0; k < 3; ++k) {
        double t = j3[k] * g.h - R[k];
        t -= L * std::nearbyint(t / L);
        dv[k] = t;
        r2 += t * t;
      }
      if (r2 < rc2) {
        inside.push_back(p);
        dd.push_back(dv[0]);
        dd.push_back(dv[1]);
        dd.push_back(dv[2]);
        dd.push_back(r2);
      }
    }
    const size_t np = inside.size();
    std::vector<double> beta(np * g.nproj);
    std::vector<double> norm(g.nproj, 0.0);
    for (size_t i = 0; i < np; ++i) {
      const double gs = std::exp(-dd[4 * i + 3] / s2);
      beta[i * g.nproj] = gs;
      if (g.nproj == 4)
        for (int k = 0; k < 3; ++k) beta[i * 4 + 1 + k] = dd[4 * i + k] * gs;
      for (int l = 0; l < g.nproj; ++l) norm[l] += beta[i * g.nproj + l] * beta[i * g.nproj + l];
    }
    for (int l = 0; l < g.nproj; ++l) {
      const double s = (norm[l] > 0) ? 1.0 / std::sqrt(g.dV * norm[l]) : 0.0;
      for (size_t i = 0; i < np; ++i) beta[i * g.nproj + l] *= s;
    }
    for (size_t i = 0; i < np; ++i) {
      g.sph_idx.push_back(inside[i]);
      g.sph_atom.push_back(a);
      for (int l = 0; l < g.nproj; ++l) g.sph_beta.push_back(beta[i * g.nproj + l]);
    }
    g.sph_off.push_back((int)g.sph_idx.size());
  }
  // inverse lists (grid point -> its sphere points, atoms in index order)
  std::map<int, std::vector<int>> cover;
  for (size_t i = 0; i < g.sph_idx.size(); ++i) cover[g.sph_idx[i]].push_back((int)i);
  g.cov_idx.clear();
  g.cov_off.assign(1, 0);
  g.cov_ent.clear();
  for (auto& kv : cover) {
    g.cov_idx.push_back(kv.first);
    for (int e : kv.second) g.cov_ent.push_back(e);
    g.cov_off.push_back((int)g.cov_ent.size());
  }

}

void build_geometry(const ks_cell_desc& d, HostGeometry& g) {
  if (d.natoms < 0 || (d.natoms > 0 && !d.pos)) fail(KS_ERR_ARG, "natoms=%d with pos=%p", d.natoms, (const void*)d.pos);
  if (d.nproj != 1 && d.nproj != 4) fail(KS_ERR_ARG, "nproj must be 1 or 4, got %d", d.nproj);
  if (d.nstates < 1) fail(KS_ERR_ARG, "nstates must be >= 1, got %d", d.nstates);
  if (!(d.vloc_width > 0) || !(d.proj_sigma > 0) || !(d.proj_rc > 0)) fail(KS_ERR_ARG, "widths and radii must be > 0");
  int nG = 0;
  count_sphere(d.L, d.N, d.ecut, &nG);
  const int N = d.N;
  const double L = d.L;
  g.L = L;
  g.N = N;
  g.ecut = d.ecut;
  g.h = L / N;
  g.omega = L * L * L;
  g.dV = g.omega / (double(N) * N * N);
  if (d.natoms > 0 && 2.0 * d.proj_rc >= L)
    fail(KS_ERR_ARG, "projector sphere diameter %g exceeds the cell %g", 2 * d.proj_rc, L);

  // ---- sphere in canonical order, with its z-columns --------------------------------------
  const double kf = 2.0 * M_PI / L;
  g.gidx.clear();
  g.mvec.clear();
  g.g2half.clear();
  g.col_xy.clear();
  g.col_off.clear();
  g.col_half.clear();
  g.xr = 0;
  for (int jx = 0; jx < N; ++jx)
    for (int jy = 0; jy < N; ++jy) {
      int cnt = 0;
      const int first = (int)g.gidx.size();
      for (int jz = 0; jz < N; ++jz) {
        const int mx = freq(jx, N), my = freq(jy, N), mz = freq(jz, N);
        const double g2 = kf * kf * double(mx * mx + my * my + mz * mz);
        if (0.5 * g2 <= d.ecut) {
          g.gidx.push_back((jx * N + jy) * N + jz);
          g.mvec.push_back(mx);
          g.mvec.push_back(my);
          g.mvec.push_back(mz);
          g.g2half.push_back(0.5 * g2);
          ++cnt;
        }
      }
      if (cnt > 0) {
        if (cnt % 2 != 1) fail(KS_ERR_ARG, "internal: even column count");
        const int hz = cnt / 2;
        // The column must be the symmetric range |m_z| <= hz.
        for (int k = 0; k < cnt; ++k) {
          const int jz = (k <= hz) ? k : N - cnt + k;
          if (g.gidx[first + k] != (jx * N + jy) * N + jz) fail(KS_ERR_ARG, "internal: column not contiguous");
        }
        g.col_xy.push_back(jx * N + jy);
        g.col_off.push_back(first);
        g.col_half.push_back(hz);
        g.xr = std::max(g.xr, std::max(std::abs(freq(jx, N)), std::abs(freq(jy, N))));
      }
    }
  g.nG = (int)g.gidx.size();
  g.ncols = (int)g.col_xy.size();
  if (g.nG != nG) fail(KS_ERR_ARG, "internal: sphere count mismatch");

  g.vloc_depth = d.vloc_depth;
  g.vloc_width = d.vloc_width;
  g.natoms = d.natoms;
  g.nproj = d.nproj;
  g.D = d.proj_D;
  g.proj_sigma = d.proj_sigma;
  g.proj_rc = d.proj_rc;
  build_atoms(d.pos, g, true);

  g.occ.assign(d.nstates, 1.0);
  if (d.occ)
    for (int k = 0; k < d.nstates; ++k) g.occ[k] = d.occ[k];

  g.tw.resize(2 * N);
  for (int t = 0; t < N; ++t) {
    g.tw[2 * t] = std::cos(2.0 * M_PI * t / N);
    g.tw[2 * t + 1] = std::sin(2.0 * M_PI * t / N);
  }
}

}  // namespace ks
