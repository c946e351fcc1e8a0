// Shared host/device definitions of the CUDA path: error handling, complex types,
// the host geometry tables.  Nothing here is shared with the oracle.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "ks.h"

namespace ks {

// ---------------------------------------------------------------------------------------------
// Errors: internal code throws ks::Error; every ABI entry point catches it and returns st.
// ---------------------------------------------------------------------------------------------
struct Error {
  ks_status st;
};

void set_last_error(const std::string& msg);
[[noreturn]] void fail(ks_status st, const char* fmt, ...);
[[noreturn]] void fail_cuda(cudaError_t e, const char* what, const char* file, int line);

#define KS_CUDA(call)                                                  \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) ks::fail_cuda(e_, #call, __FILE__, __LINE__); \
  } while (0)

// Every kernel launch is followed by KS_CHECK_LAUNCH(): it counts the launch (reported by
// ks_kernel_launches) and turns a launch error into ks::Error.
void note_launch();
#define KS_CHECK_LAUNCH()          \
  do {                             \
    ks::note_launch();             \
    KS_CUDA(cudaGetLastError());   \
  } while (0)

// ---------------------------------------------------------------------------------------------
// Complex types: float2 / double2 with the few operations the kernels use.
// ---------------------------------------------------------------------------------------------
template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cplx = typename cplx_of<T>::type;

template <typename C> __host__ __device__ __forceinline__ C mk(decltype(C::x) r, decltype(C::x) i) {
  C c;
  c.x = r;
  c.y = i;
  return c;
}
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 operator*(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator*(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
  return mk<C>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// ---------------------------------------------------------------------------------------------
// Host geometry: cutoff sphere, z-columns, V_loc, projector spheres (built once per handle).
// ---------------------------------------------------------------------------------------------
struct HostGeometry {
  double L = 0, h = 0, omega = 0, dV = 0, ecut = 0;
  int N = 0, nG = 0;
  std::vector<int> gidx;        // packed G -> flat grid index (jx*N + jy)*N + jz
  std::vector<int> mvec;        // [nG][3] integer frequencies
  std::vector<double> g2half;   // |G|^2 / 2
  // z-columns of the sphere: a column (jx, jy) holds cnt = 2*hz+1 consecutive packed
  // entries; entry k sits at jz = k (k <= hz) or jz = N - cnt + k (k > hz).
  int ncols = 0;
  std::vector<int> col_xy;      // jx*N + jy, increasing
  std::vector<int> col_off;     // first packed index of the column
  std::vector<int> col_half;    // hz
  int xr = 0;                   // columns exist only for |m_x| <= xr (and |m_y| <= xr)
  double vmin = 0, vmax = 0;     // extremes of V_loc (formed on the device)
  std::vector<double> pos;      // [natoms][3] atom positions (bohr)
  double vloc_depth = 0, vloc_width = 0;
  // projectors: sphere point lists per atom (grid order within an atom)
  int natoms = 0, nproj = 0;
  double D = 0, proj_sigma = 0, proj_rc = 0;
  std::vector<int> sph_off;     // [natoms+1]
  std::vector<int> sph_idx;     // flat grid index of each sphere point
  std::vector<int> sph_atom;    // atom of each sphere point
  std::vector<double> sph_beta; // [npts][nproj]
  std::vector<int> sph_zorder;  // [npts] the atom's sphere points visited plane by plane (z, then x, y)
  // inverse lists: every grid point covered by >= 1 sphere, with its sphere points in atom order
  std::vector<int> cov_idx;     // flat grid index, increasing
  std::vector<int> cov_off;     // [ncov+1]
  std::vector<int> cov_ent;     // sphere point indices
  std::vector<int> cov_scratch; // [N^3 + 1] counts, kept between rebuilds (no page faults per move)
  std::vector<double> occ;      // [nstates]
  std::vector<double> tw;       // [N][2] cos, sin of 2 pi t / N
};

bool valid_fft_length(int N);
void count_sphere(double L, int N, double ecut, int* nG);
void build_geometry(const ks_cell_desc& d, HostGeometry& g);
// Rebuilds the atom-dependent parts (pos, the projector sphere lists and their inverse lists)
// for new positions pos [natoms][3] of the same atoms.  V_loc, vmin and vmax are the
// engine's to fill (on the device).
void build_atoms(const double* pos, HostGeometry& g);

}  // namespace ks
