// Host-side setup of one cell: the plane-wave cutoff sphere and its z-columns, the local
// potential on the grid, and the real-space projector spheres (Sec. "Pseudopotentials",
// Eq. 9).  Built once per handle in FP64 and copied to the device.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <thread>

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

void build_atoms(const double* pos, HostGeometry& g) {
  const int N = g.N;
  const double L = g.L;
  // V_loc (the 27-image Gaussians of Sec. "Pseudopotentials") is formed on the device from
  // separable per-axis factors; only its extremes are kept on the host.
  g.pos.assign(pos ? pos : nullptr, pos ? pos + 3 * (size_t)g.natoms : nullptr);

  // ---- projector spheres |d| < R_c around each atom (minimum image), grid order ----------
  // Atoms are independent: threads take contiguous ranges of atoms and the per-atom lists are
  // joined in atom order, so the result does not depend on the thread count.
  const double s2 = 2.0 * g.proj_sigma * g.proj_sigma;
  const double rc2 = g.proj_rc * g.proj_rc;
  struct AtomPts {
    std::vector<int> idx;
    std::vector<double> beta;
    std::vector<int> zorder;                                          // positions in idx
  };
  std::vector<AtomPts> per(g.natoms);
  auto one_atom = [&](int a) {
    const double R[3] = {pos[3 * a], pos[3 * a + 1], pos[3 * a + 2]};
    int lo[3], hi[3];
    // per axis: wrapped grid index and minimum-image displacement of each box coordinate
    std::vector<int> jw[3];
    std::vector<double> dw[3];
    for (int k = 0; k < 3; ++k) {
      lo[k] = (int)std::floor((R[k] - g.proj_rc) / g.h) - 1;
      hi[k] = (int)std::ceil((R[k] + g.proj_rc) / g.h) + 1;
      for (int i = lo[k]; i <= hi[k]; ++i) {
        const int j = ((i % N) + N) % N;
        double t = j * g.h - R[k];
        t -= L * std::nearbyint(t / L);
        jw[k].push_back(j);
        dw[k].push_back(t);
      }
    }
    // box points inside the sphere, then in grid order (a box wider than the grid would
    // repeat an index: the repeats are dropped)
    std::vector<std::pair<int, int>> hit;                            // (grid index, slot in cand)
    std::vector<double> cand;                                         // dx, dy, dz, r2 per hit
    for (size_t ix = 0; ix < jw[0].size(); ++ix)
      for (size_t iy = 0; iy < jw[1].size(); ++iy)
        for (size_t iz = 0; iz < jw[2].size(); ++iz) {
          const double dx = dw[0][ix], dy = dw[1][iy], dz = dw[2][iz];
          const double r2 = dx * dx + dy * dy + dz * dz;
          if (!(r2 < rc2)) continue;
          hit.push_back({(jw[0][ix] * N + jw[1][iy]) * N + jw[2][iz], (int)(cand.size() / 4)});
          cand.insert(cand.end(), {dx, dy, dz, r2});
        }
    // a box inside [0, N) on every axis enumerates in grid order already
    bool wraps = false;
    for (int k = 0; k < 3; ++k) wraps = wraps || lo[k] < 0 || hi[k] >= N;
    if (wraps) std::sort(hit.begin(), hit.end());
    AtomPts& out = per[a];
    std::vector<double> dd;
    for (size_t i = 0; i < hit.size(); ++i) {
      if (i > 0 && hit[i].first == hit[i - 1].first) continue;
      out.idx.push_back(hit[i].first);
      dd.insert(dd.end(), cand.begin() + 4 * hit[i].second, cand.begin() + 4 * hit[i].second + 4);
    }
    const size_t np = out.idx.size();
    std::vector<double>& beta = out.beta;
    beta.assign(np * g.nproj, 0.0);
    std::vector<double> norm(g.nproj, 0.0);
    for (size_t i = 0; i < np; ++i) {
      const double gs = std::exp(-dd[4 * i + 3] / s2);
      beta[i * g.nproj] = gs;
      if (g.nproj == 4)
        for (int k = 0; k < 3; ++k) beta[i * 4 + 1 + k] = dd[4 * i + k] * gs;
      for (int l = 0; l < g.nproj; ++l) norm[l] += beta[i * g.nproj + l] * beta[i * g.nproj + l];
    }
    for (int l = 0; l < g.nproj; ++l) {
      const double sc = (norm[l] > 0) ? 1.0 / std::sqrt(g.dV * norm[l]) : 0.0;
      for (size_t i = 0; i < np; ++i) beta[i * g.nproj + l] *= sc;
    }
    // plane-major visiting order (box z outermost, then x, then y): a pass over a grid laid
    // out [z][x][y] then reads runs of consecutive y (a grid index met twice, in a box wider
    // than the grid, is visited once)
    std::vector<char> seen(np, 0);
    for (size_t iz = 0; iz < jw[2].size(); ++iz)
      for (size_t ix = 0; ix < jw[0].size(); ++ix)
        for (size_t iy = 0; iy < jw[1].size(); ++iy) {
          const double dx = dw[0][ix], dy = dw[1][iy], dz = dw[2][iz];
          if (!(dx * dx + dy * dy + dz * dz < rc2)) continue;
          const int gi = (jw[0][ix] * N + jw[1][iy]) * N + jw[2][iz];
          const auto it = std::lower_bound(out.idx.begin(), out.idx.end(), gi);
          const int q = (int)(it - out.idx.begin());
          if (!seen[q]) {
            seen[q] = 1;
            out.zorder.push_back(q);
          }
        }
  };
  const int nthr = (int)std::max(1, std::min<int>({8, g.natoms / 8, (int)std::thread::hardware_concurrency()}));
  if (nthr > 1) {
    std::vector<std::thread> pool;
    for (int t = 0; t < nthr; ++t)
      pool.emplace_back([&, t] {
        for (int a = (int)((long)g.natoms * t / nthr); a < (int)((long)g.natoms * (t + 1) / nthr); ++a) one_atom(a);
      });
    for (auto& th : pool) th.join();
  } else {
    for (int a = 0; a < g.natoms; ++a) one_atom(a);
  }
  g.sph_off.assign(1, 0);
  g.sph_idx.clear();
  g.sph_atom.clear();
  g.sph_beta.clear();
  g.sph_zorder.clear();
  for (int a = 0; a < g.natoms; ++a) {
    const int base = (int)g.sph_idx.size();
    for (int q : per[a].zorder) g.sph_zorder.push_back(base + q);
    g.sph_idx.insert(g.sph_idx.end(), per[a].idx.begin(), per[a].idx.end());
    g.sph_atom.insert(g.sph_atom.end(), per[a].idx.size(), a);
    g.sph_beta.insert(g.sph_beta.end(), per[a].beta.begin(), per[a].beta.end());
    g.sph_off.push_back((int)g.sph_idx.size());
  }
  // inverse lists (grid point -> its sphere points, atoms in index order): count the sphere
  // points of every grid point, then place the points in increasing order
  const size_t N3 = (size_t)N * N * N;
  std::vector<int>& first = g.cov_scratch;
  first.resize(N3 + 1);
  std::fill(first.begin(), first.end(), 0);
  for (int idx : g.sph_idx) ++first[idx + 1];
  g.cov_idx.clear();
  g.cov_off.assign(1, 0);
  for (size_t j = 0; j < N3; ++j) {
    if (first[j + 1] > 0) {
      g.cov_idx.push_back((int)j);
      g.cov_off.push_back(g.cov_off.back() + first[j + 1]);
    }
    first[j + 1] += first[j];                                         // first[j]: start of point j's entries
  }
  g.cov_ent.assign(g.sph_idx.size(), 0);
  for (size_t i = 0; i < g.sph_idx.size(); ++i) g.cov_ent[first[g.sph_idx[i]]++] = (int)i;

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
  build_atoms(d.pos, g);

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
