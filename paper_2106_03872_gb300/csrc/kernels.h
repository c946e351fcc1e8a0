// Launchers of the CUDA kernels (one per kernel), templated on the real type T
// (float: mixed path, double: FP64 path).  All launches are asynchronous on `s`.
#pragma once

#include "common.h"

namespace ks {

// Raw device views of one cell's tables.
template <typename T> struct DevTables {
  int N = 0, nG = 0, ncols = 0, natoms = 0, nproj = 0, ncov = 0, xr = 0;
  double L = 0, omega = 0, dV = 0, D = 0;
  const int* gidx = nullptr;          // [nG]
  const T* g2half = nullptr;          // [nG]
  const cplx<T>* tw = nullptr;        // [N] exp(+2 pi i t/N)
  const int* col_xy = nullptr;        // [ncols]
  const int* col_off = nullptr;       // [ncols]
  const int* col_half = nullptr;      // [ncols]
  const int* sph_off = nullptr;       // [natoms+1]
  const int* sph_idx = nullptr;       // [npts]
  const int* sph_atom = nullptr;      // [npts]
  const T* sph_beta = nullptr;        // [npts][nproj]
  const int* sph_zorder = nullptr;    // [npts] plane-major visiting order of each atom's points
  const int* cov_idx = nullptr;       // [ncov]
  const int* cov_off = nullptr;       // [ncov+1]
  const int* cov_ent = nullptr;       // [nent]
};

// ---- full-grid (plain) path --------------------------------------------------------------------
// In-place batched 1D FFTs along one axis (0: x, 1: y, 2: z) of nb grids [N][N][N].
template <typename T> void fft_axis(cplx<T>* grid, int nb, int N, int axis, int sign, const cplx<T>* tw, cudaStream_t s);
// grid[b][gidx[g]] = psi[b][g] (grid must be zeroed before).
template <typename T> void scatter_sphere(const cplx<T>* psi, cplx<T>* grid, const DevTables<T>& t, int nb, cudaStream_t s);
// hpsi[b][g] = scale * grid[b][gidx[g]] + g2half[g] * psi[b][g] (no kinetic term if psi is null)
template <typename T> void gather_kinetic(const cplx<T>* grid, const cplx<T>* psi, cplx<T>* hpsi, const DevTables<T>& t,
                                          int nb, T scale, cudaStream_t s);
// grid[b][j] *= v[j]
template <typename T> void multiply_potential(cplx<T>* grid, const T* v, int N3, int nb, cudaStream_t s);
// one grid [N][N][N]: grid[j] *= exp(i kappa . (r_j - L/2)), r_j = (L/N) (jx, jy, jz)
template <typename T> void multiply_phase(cplx<T>* grid, int N, double L, const double kappa[3], cudaStream_t s);
// Forces (Eq. 11): grid[b][gidx[g]] = i G_alpha c_bg for nb states (grids zeroed before)
template <typename T> void scatter_grad(const cplx<T>* psi, cplx<T>* grid, const DevTables<T>& t, int alpha, int nb,
                                        cudaStream_t s);
// gacc[j] += sum_{b < nb} occ[b] 2 Re(conj(dpsi[b][j]) psi[b][j])  (states in order, summed in T)
template <typename T> void grad_accumulate(const cplx<T>* dpsi, const cplx<T>* psi, T* gacc, int N3, int nb,
                                           const double* occ, cudaStream_t s);
// fnl[3 I + alpha] -= w sum_{b < nb} occ[b] sum_l Re(conj(q_bIl) p_bIl) (projections [nb][natoms][nproj])
template <typename T> void nl_force(const cplx<T>* p, const cplx<T>* q, int natoms, int nproj, int nb, double w,
                                    const double* occ, double* fnl, int alpha, cudaStream_t s);
// floc[3 I + a] = coef sum_j X_I[jx] Y_I[jy] Z_I[jz] g_a[j], g [3][N^3], xyz [natoms][3][N];
// zmajor: g laid out [z][x][y].  Each atom's sum runs over LOCAL_FORCE_SPLIT slices of the
// grid (partials [natoms][LOCAL_FORCE_SPLIT][3]), then the slices are added in order.
constexpr int LOCAL_FORCE_SPLIT = 8;
template <typename T> void local_force(const T* g, const double* xyz, int N, int natoms, double coef, double* partials,
                                       double* floc, cudaStream_t s, bool zmajor = false);
// out[b][g] = i G_alpha c_bg (packed, nb states)
template <typename T> void grad_packed(const cplx<T>* psi, cplx<T>* out, const DevTables<T>& t, int alpha, int nb,
                                       cudaStream_t s);
// out[0] = min_j v[j], out[1] = max_j v[j] (device); partials holds 2 * nblocks doubles
void minmax(const double* v, size_t n, double* partials, int nblocks, double* out, cudaStream_t s);
// v[j] = depth sum_I X_I[jx] Y_I[jy] Z_I[jz] (xyz as for local_force), in FP64; v64 (may be
// NULL) receives the FP64 values
template <typename T> void vloc_from_axes(const double* xyz, int natoms, int N, double depth, T* v, double* v64,
                                          cudaStream_t s);
// out[3] (device) = dV sum_j n_j (r_j - L/2); partials holds nblocks * 3 doubles
template <typename T> void dipole(const T* n, int N, double L, double* partials, int nblocks, double* out,
                                  cudaStream_t s);
// proj[b][I][l] = scale * sum_{j in sphere I} beta_Il(j) grid[b][j]
// zmajor: the grids are laid out [b][z][x][y] (the fused path's real-space planes)
template <typename T> void nl_project(const cplx<T>* grid, const DevTables<T>& t, cplx<T>* proj, int nb, T scale, cudaStream_t s,
                                      bool zmajor = false);
// grid[b][j] += scale * sum_{(I,l) covering j} beta_Il(j) proj[b][I][l]
template <typename T> void nl_add(cplx<T>* grid, const DevTables<T>& t, const cplx<T>* proj, int nb, T scale, cudaStream_t s);
// n[j] (+)= scale * sum_b occ[b] |grid[b][j]|^2 (states in order; first batch overwrites)
template <typename T> void density_accumulate(const cplx<T>* grid, const double* occ, T* n, int N3, int nb, T scale,
                                              bool first, cudaStream_t s);

// ---- potentials and reductions --------------------------------------------------------------
// work[j] = n[j] (complex)
template <typename T> void real_to_complex(const T* n, cplx<T>* work, int N3, cudaStream_t s);
// work(G) *= 4 pi / |G|^2 * scale, 0 at G = 0 (full-grid FFT order)
template <typename T> void poisson_multiply(cplx<T>* work, int N, double L, T scale, cudaStream_t s);
// vtot = vloc + Re(work) + v_x(n); partials[blk][3] of (n v_H, n eps_x, n v_x) sums
template <typename T> void hxc_combine(const T* n, const cplx<T>* work, const T* vloc, T* vtot, double* partials,
                                       int N3, int nblocks, cudaStream_t s);
// parts[0..2] = dV * (0.5 sum n vH, sum n eps_x, sum n v_x) from the partials
void hxc_finish(const double* partials, int nblocks, double dV, double* parts, cudaStream_t s);
// nin <- nin + mix (nout - nin) over N3 points; partials[b] (nblocks) = sum of |nout - nin| before
// the update in block b.  sum_partials: *out = scale * sum_b partials[b] (fixed order).
template <typename T> void density_mix(const T* nout, T* nin, int N3, double mix, double* partials, int nblocks,
                                       cudaStream_t s);
void sum_partials(const double* partials, int nblocks, double scale, double* out, cudaStream_t s);
// History mixing of the density (Pulay / DIIS and Broyden): at most PULAY_MAX (n_in, R) pairs.
constexpr int PULAY_MAX = 8;
template <typename T> struct PulayRefs {
  const T* r[PULAY_MAX];   // the other history residuals
  int m;
};
template <typename T> struct PulayMix {
  const T* n[PULAY_MAX];
  const T* r[PULAY_MAX];
  double a[PULAY_MAX];     // coefficients of n_q
  double b[PULAY_MAX];     // coefficients of r_q
  int m;
};
// hr = nout - nin, hn = nin; out (device, 2 + PULAY_MAX) = dV * {sum |R|, sum R^2, sum R r_q};
// partials holds nblocks * (2 + PULAY_MAX) doubles
template <typename T> void pulay_store(const T* nout, const T* nin, T* hn, T* hr, int N3, const PulayRefs<T>& refs,
                                       double* partials, int nblocks, double dV, double* out, cudaStream_t s);
// nin = sum_i a_i n_i + b_i r_i
template <typename T> void pulay_mix(T* nin, int N3, const PulayMix<T>& p, cudaStream_t s);
// Teter-preconditioned SD update of n states [n][nG]: R = hpsi - eig psi, T_b = kinetic energy
// of R_b (sum g2half |R|^2 / sum |R|^2) floored at tmin, psi_b -= K(g2half / T_b) R_b / (T_b + shift).
// trr (device, n double2) receives (sum g2half |R|^2, sum |R|^2) per state.
template <typename T> void teter_update(cplx<T>* psi, const cplx<T>* hpsi, const T* g2half, const double* eig,
                                        double2* trr, double shift, double tmin, int nG, int n, cudaStream_t s);
constexpr int HXC_BLOCKS = 296;

// dots[b] = sum_g conj(a[b][g]) b[b][g] (FP64 accumulation, fixed order)
template <typename T> void state_dots(const cplx<T>* a, const cplx<T>* b, int nG, int nb, double2* dots, cudaStream_t s);
// out[0] = sum_b occ[b] Re(dots[b]) - parts[0] + parts[1] - parts[2]   (parts may be NULL)
void weighted_energy(const double2* dots, const double* occ, int nb, const double* parts, double* out, cudaStream_t s);

// acc1 += a1 * w; acc2 += a2 * w  (complex constants; acc2 may be NULL).  With base non-NULL
// the accumulators start from it instead: acc1 = base + a1 w, acc2 = base + a2 w.
template <typename T> void axpy2(cplx<T>* acc1, double2 a1, cplx<T>* acc2, double2 a2, const cplx<T>* w,
                                 const cplx<T>* base, size_t n, cudaStream_t s);
// psi[b][g] = seeded uniform(-0.5, 0.5) + i uniform(-0.5, 0.5)
template <typename T> void random_states(cplx<T>* psi, size_t n, uint64_t seed, cudaStream_t s);
// complex128 <-> internal precision
template <typename T> void from_c128(const double2* in, cplx<T>* out, size_t n, cudaStream_t s);
template <typename T> void to_c128(const cplx<T>* in, double2* out, size_t n, cudaStream_t s);
template <typename T> void real_to_double(const T* in, double* out, size_t n, cudaStream_t s);

// ---- dense linear algebra (dense.cu) ----------------------------------------------------------
// out[i][j] = sum_k conj(A[i][k]) B[j][k] for i < m, j < n (row-major, FP64 out); split-K with
// deterministic reduction through `part` (>= gemm_cn_parts(...) double2 elements).
template <typename T> void gemm_cn(const cplx<T>* A, int lda, const cplx<T>* B, int ldb, int m, int n, int K,
                                   double2* part, size_t part_elems, double2* out, cudaStream_t s);
// Y[i][k] = sum_j M[i][j] X[j][k], i < m, j < nin, k < K; rows j >= nin1 of X come from X2
// (row j - nin1) when X2 is non-NULL.  Y must not overlap X or X2.
template <typename T> void rotate(const double2* M, int nin, const cplx<T>* X, const cplx<T>* X2, int nin1, int ldx,
                                  cplx<T>* Y, int ldy, int m, int K, cudaStream_t s);
// A := (A + A^H)/2
void hermitize(double2* A, int n, cudaStream_t s);
// C = opA(A) opB(B), n x n complex128 (row-major); flags: 1 conj(A), 2 B transposed, 4 conj(B).
// mixed: FP32 products within 32-wide K chunks, FP64 chunk sums; else FP64.
constexpr int SP_CONJ_A = 1, SP_TRANS_B = 2, SP_CONJ_B = 4;
void small_product(const double2* A, const double2* B, int n, int flags, bool mixed, double2* C, cudaStream_t s);
// Mcat [n][2n] = [ (I + alpha diag(eig)) C | -alpha C ]
void sd_matrix(const double2* C, const double* eig, double alpha, int n, double2* Mcat, cudaStream_t s);
// Cholesky S = L L^H of A (in place, lower) then M = conj(L^{-1}); on failure status = 1 and
// M = I.  FP64, one CTA.
void cholesky_inverse(double2* A, double2* M, int n, int* status, cudaStream_t s);
// Same with an explicit relative pivot tolerance (pivot <= tol * S_jj fails).
void cholesky_inverse_tol(double2* A, double2* M, int n, double tol, int* status, cudaStream_t s);
// Mixed path (n <= 160): M = conj(L^{-1}) for S = L L^H from an FP32 Cholesky pass, refined
// by FP64 triangular products when `refine` (cholqr_mixed.cu); work holds
// cholesky_mixed_workspace(n) complex128.  M32, when given, receives an FP32 copy of M.
// Same status convention as cholesky_inverse.
size_t cholesky_mixed_workspace(int n);
void cholesky_inverse_mixed(const double2* S, double2* M, int n, double tol, double2* work, int* status,
                            cudaStream_t s, float2* M32 = nullptr, bool refine = true);
// Hermitian eigen-decomposition of A (destroyed) by cyclic Jacobi; eig ascending, rows of
// Vt = eigenvectors (largest-magnitude component real positive).  `V` is n*n workspace.
void jacobi_eigh(double2* A, double2* V, double* eig, double2* Vt, int n, cudaStream_t s);
// Householder + bisection + twisted-factorization eigenvectors, FP32, one CTA (n <= 128):
// V (n x n complex128, columns = eigenvectors, unsorted).
void eigh_householder_f32(const double2* A, double2* V, int n, cudaStream_t s);
// Mixed path (n <= 128): eigh_householder_f32 on the FP64 Hermitian A (kept), eigenvalues =
// FP64 Rayleigh quotients of the FP32 vectors on A; same outputs as jacobi_eigh.
// V is n*n workspace, lam n doubles of workspace.
void eigh_mixed(const double2* A, double2* V, double* lam, double* eig, double2* Vt, int n, cudaStream_t s);
// Mixed path for 128 < n <= 256: FP32 parallel Jacobi on a copy of A (one CTA, matrix in
// global memory), eigenvalues = FP64 Rayleigh quotients of the FP32 vectors on A; same outputs
// as eigh_mixed.  work: 2 n^2 complex64.
void eigh_jacobi_mixed(const double2* A, double2* V, double* lam, double* eig, double2* Vt, float2* work, int n,
                       cudaStream_t s);
// Rayleigh-Ritz step of the mixed block iteration in one CTA (n <= 128), FP32 in and out:
// H_sub = conj(M) Hraw M^T (Hermitian part, exported to Aout), its eigenpairs, C = Vt M and
// Mcat = [(I + alpha Lambda) C | -alpha C] (n x 2n) with rows in ascending eigenvalue order;
// Vout holds the eigenvectors as columns in solver order and perm their ranks.
void rr_step_mixed(const float2* Hraw, const float2* M, double alpha, int n, float2* Mcat, float2* Aout,
                   float2* Vout, int* perm, cudaStream_t s);
// eig[perm[j]] = FP64 Rayleigh quotient of column j of V on A (outputs of rr_step_mixed).
void ritz_values(const float2* A, const float2* V, const int* perm, int n, double* eig, cudaStream_t s);

// ---- tensor-core GEMMs (tc_gemm.cu), split-BF16 (hi*hi + hi*lo + lo*hi), FP32 accumulation ---------
// Same contract as gemm_cn<float> / rotate<float>; err receives 1 if a bounded wait expired.
// out32, when given, receives an FP32 copy of out.  Aimg, when given, is A's pre-split image
// (tc_overlap_prepare_a of the same A, m and K): A's operand tiles then arrive by bulk copy.
void tc_overlap(const float2* A, int lda, const float2* B, int ldb, int m, int n, int K, double2* part,
                size_t part_elems, double2* out, int* err, cudaStream_t s, float2* out32 = nullptr,
                const void* Aimg = nullptr);
// Bytes of the pre-split image of an m x K operand, and the image itself (bf16 hi and lo
// operand tiles per 128-row tile and chunk of 16 complex; a constant operand is split once).
size_t tc_overlap_image_bytes(int m, int K);
void tc_overlap_prepare_a(const float2* A, int lda, int m, int K, void* img, cudaStream_t s);
// Partial-buffer elements tc_overlap wants for an m x n output (one wave of CTAs).
size_t tc_overlap_part_elems(int m, int n, bool prepared = false);
void tc_rotate(const double2* M, int nin, const float2* X, const float2* X2, int nin1, int ldx, float2* Y, int ldy,
               int m, int K, void* work, size_t work_bytes, int* err, cudaStream_t s);
size_t tc_rotation_workspace_bytes(int m, int nin);
// tc_rotate in two steps, for one FP32 M applied to several blocks: split M (m x nin) into the
// workspace once, then run rotations from it.
void tc_rotate_prepare(const float2* M, int m, int nin, void* work, size_t work_bytes, cudaStream_t s);
void tc_rotate_prepared(const void* work, int nin, const float2* X, const float2* X2, int nin1, int ldx, float2* Y,
                        int ldy, int m, int K, int* err, cudaStream_t s);

}  // namespace ks
