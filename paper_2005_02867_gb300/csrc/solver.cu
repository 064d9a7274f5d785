// Linear solvers of the step: Jacobi-preconditioned CG for the energy,
// species and momentum systems, and CG preconditioned by a symmetric
// geometric multigrid V-cycle for the variable-density pressure equation
// (Eq. pequation).  Dot products and the CG scalars are FP64; the multigrid
// hierarchy is FP64 or FP32.  Convergence is tested on the device: every
// kernel of an iteration returns at once when the done flag is set, so the
// host only reads the status every few iterations.
#include <cstdio>
#include <cstring>
#include <algorithm>
#include "kernels.h"

namespace dg {

// (S_ITSK: the iterations of each system of a joint persistent solve)
// S_TMO: 1 when a grid-barrier wait of the last persistent solve ran out (written by the
// last block to leave the launch)
// S_SCL: the power of two that brings the initial defect's norm into [2^-100, 2^100]
// (1 when it is there), by which the binary32 defect-correction solve scales its defect
enum { S_RZ = 0, S_PAP, S_RR, S_BB, S_ALPHA, S_BETA, S_ITS, S_TOL2, S_MAXIT, S_ITSK, S_TMO = S_ITSK + 3, S_SCL,
       S_ISCL, S_COUNT };   // S_ISCL = 1 / S_SCL

// done flag values: 0 running, 1 converged, 2 stopped at the iteration cap

struct BoxV {
  int m[3];
  long long N;
  const double* D;
  const double* c[3];
};

__device__ __forceinline__ void bdecomp(const int m[3], long long id, int& i, int& j, int& k) {
  unsigned u = (unsigned)id;
  unsigned t = u / (unsigned)m[0];
  i = (int)(u - t * (unsigned)m[0]);
  unsigned t2 = t / (unsigned)m[1];
  j = (int)(t - t2 * (unsigned)m[1]);
  k = (int)t2;
}

// y = A x at cell id, and the total diagonal D + sum of adjacent couplings
template <typename T, typename TX, bool DT = true>
__device__ __forceinline__ void box_row(const int m[3], const T* D, const T* const c[3], const TX* x, long long id,
                                        int i, int j, int k, double& ax, double& dtot) {
  double xp = (double)x[id];
  double y = (double)D[id] * xp;
  double dt = (double)D[id];
  int q[3] = {i, j, k};
  long long st[3] = {1, (long long)m[0], (long long)m[0] * m[1]};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!c[a] || m[a] < 2) continue;
    if (q[a] > 0) {
      double cl = (double)c[a][id];
      y += cl * (xp - (double)x[id - st[a]]);
      if (DT) dt += cl;
    }
    if (q[a] < m[a] - 1) {
      double ch = (double)c[a][id + st[a]];
      y += ch * (xp - (double)x[id + st[a]]);
      if (DT) dt += ch;
    }
  }
  ax = y;
  dtot = dt;
}

// y = A x at cell id in the diagonal form a_P x_P - sum c x_N, a_P = D + sum of the
// adjacent couplings formed once per solve: one multiply and one FMA per neighbour, against
// a subtraction and an FMA per neighbour in the difference form (the binary64 pipe is the
// bound of an FP64 stencil on GB300; the bytes are the same, a_P read in place of D)
__device__ __forceinline__ double box_offdiag(const int m[3], const double* const c[3], const double* x,
                                              long long id, int i, int j, int k, double y) {
  const int q[3] = {i, j, k};
  const long long st[3] = {1, (long long)m[0], (long long)m[0] * m[1]};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!c[a] || m[a] < 2) continue;
    if (q[a] > 0) y = fma(-c[a][id], x[id - st[a]], y);
    if (q[a] < m[a] - 1) y = fma(-c[a][id + st[a]], x[id + st[a]], y);
  }
  return y;
}

__device__ __forceinline__ double box_row_diag(const int m[3], const double* ad, const double* const c[3],
                                               const double* x, long long id, int i, int j, int k) {
  return box_offdiag(m, c, x, id, i, j, k, ad[id] * x[id]);
}

// the total diagonal D + sum of the adjacent couplings, summed in the order of box_row
__device__ __forceinline__ double box_diag_total(const int m[3], const double* D, const double* const c[3],
                                                 long long id, int i, int j, int k) {
  double dt = D[id];
  const int q[3] = {i, j, k};
  const long long st[3] = {1, (long long)m[0], (long long)m[0] * m[1]};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!c[a] || m[a] < 2) continue;
    if (q[a] > 0) dt += c[a][id];
    if (q[a] < m[a] - 1) dt += c[a][id + st[a]];
  }
  return dt;
}

// ---------------------------------------------------------------- CG kernels
// (adg, when given, receives the total diagonal D + sum of adjacent couplings, for the
// diagonal form of the operator in k_spmv_dot)
__global__ void __launch_bounds__(TPB, Solver::CG_BLOCKS_PER_SM) k_pcg_init(BoxV A, const double* b, const double* x, double* r, double* z, double* p, double* idg,
                           int jacobi, double* part, double* adg = nullptr) {
  double acc[3] = {0, 0, 0};   // r.z, b.b, r.r
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < A.N; id += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    bdecomp(A.m, id, i, j, k);
    double ax, dt;
    if (adg) {
      // the diagonal form of the iterations (the residual recurrence then starts from the
      // operator it continues with), and the reciprocal of the diagonal by rcp64: fewer
      // binary64 instructions than the difference form and a division
      dt = box_diag_total(A.m, A.D, A.c, id, i, j, k);
      adg[id] = dt;
      ax = box_offdiag(A.m, A.c, x, id, i, j, k, dt * x[id]);
    } else {
      box_row<double, double>(A.m, A.D, A.c, x, id, i, j, k, ax, dt);
    }
    double rr = b[id] - ax;
    r[id] = rr;
    double bb = b[id];
    acc[1] += bb * bb;
    acc[2] += rr * rr;
    if (jacobi) {
      double iv = adg ? rcp64(dt) : 1.0 / dt;
      idg[id] = iv;
      double zz = iv * rr;
      z[id] = zz;
      p[id] = zz;
      acc[0] += rr * zz;
    }
  }
  block_sum_store<3>(acc, part);
}

__global__ void k_fin_init(const double* part, int nblk, double* sc, int* done, double tol2, int maxit,
                           unsigned* bar, int* err) {
  if (bar && threadIdx.x == 0) {   // grid barrier of the persistent solver back to its idle state
    bar[0] = 0u;
    bar[1] = 0u;
    *err = 0;
  }
  double rz = block_sum_partials(part, nblk);
  __syncthreads();
  double bb = block_sum_partials(part + nblk, nblk);
  __syncthreads();
  double rr = block_sum_partials(part + 2 * nblk, nblk);
  if (threadIdx.x == 0) {
    sc[S_RZ] = rz;
    sc[S_BB] = bb;
    sc[S_RR] = rr;
    sc[S_ITS] = 0.0;
    sc[S_TOL2] = tol2;
    sc[S_MAXIT] = (double)maxit;
    const double n0 = sqrt(rr);
    const bool keep = (n0 >= 0x1p-100 && n0 <= 0x1p100) || !(n0 > 0.0) || !(n0 < 1e300);
    sc[S_SCL] = keep ? 1.0 : ldexp(1.0, -ilogb(n0));
    sc[S_ISCL] = keep ? 1.0 : ldexp(1.0, ilogb(n0));
    *done = (bb == 0.0 || rr <= tol2 * bb) ? 1 : 0;
  }
}

// Ap = A p and p.Ap; with a counter (cnt != null) the last block also sets alpha = rz / pAp.
// adg (the total diagonal from k_pcg_init) selects the diagonal form of the operator.
__global__ void __launch_bounds__(TPB, Solver::CG_BLOCKS_PER_SM) k_spmv_dot(BoxV A, const double* p, double* Ap, double* part, const int* done, double* sc,
                           unsigned* cnt, const double* adg = nullptr) {
  if (*done) return;
  double acc[1] = {0.0};
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < A.N; id += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    bdecomp(A.m, id, i, j, k);
    double ax;
    if (adg) {
      ax = box_row_diag(A.m, adg, A.c, p, id, i, j, k);
    } else {
      double dt;
      box_row<double, double, false>(A.m, A.D, A.c, p, id, i, j, k, ax, dt);
    }
    Ap[id] = ax;
    acc[0] += p[id] * ax;
  }
  block_sum_store<1>(acc, part);
  if (cnt && last_block(cnt)) {
    double pap = block_sum_partials(part, gridDim.x);
    if (threadIdx.x == 0) {
      sc[S_PAP] = pap;
      sc[S_ALPHA] = sc[S_RZ] / pap;
      *cnt = 0u;
    }
  }
}

__global__ void k_fin_alpha(const double* part, int nblk, double* sc, const int* done) {
  if (*done) return;
  double pap = block_sum_partials(part, nblk);
  if (threadIdx.x == 0) {
    sc[S_PAP] = pap;
    sc[S_ALPHA] = sc[S_RZ] / pap;
  }
}

// x += alpha p, r -= alpha Ap; Jacobi: z = r / diag and r.z; both: r.r.  bf (optional): the
// new r rounded to FP32 as the right-hand side of an FP32 multigrid's level 0
__global__ void __launch_bounds__(TPB, Solver::CG_BLOCKS_PER_SM) k_update(long long N, double* x, double* r, const double* p, const double* Ap, const double* idg,
                         double* z, int jacobi, double* sc, double* part, int* done, unsigned* cnt,
                         float* bf = nullptr) {
  if (*done) return;
  double al = sc[S_ALPHA];
  double acc[2] = {0, 0};
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < N; id += (long long)gridDim.x * blockDim.x) {
    x[id] += al * p[id];
    double rr = r[id] - al * Ap[id];
    r[id] = rr;
    if (bf) bf[id] = (float)rr;
    acc[1] += rr * rr;
    if (jacobi) {
      double zz = idg[id] * rr;
      z[id] = zz;
      acc[0] += rr * zz;
    }
  }
  block_sum_store<2>(acc, part);
  if (cnt && last_block(cnt)) {
    // iteration count, convergence test, and (Jacobi) beta: the work of k_fin_iter
    double rz = block_sum_partials(part, gridDim.x);
    __syncthreads();
    double rr = block_sum_partials(part + gridDim.x, gridDim.x);
    if (threadIdx.x == 0) {
      sc[S_ITS] += 1.0;
      sc[S_RR] = rr;
      if (rr <= sc[S_TOL2] * sc[S_BB]) *done = 1;
      else if (sc[S_ITS] >= sc[S_MAXIT]) *done = 2;
      if (jacobi) {
        sc[S_BETA] = rz / sc[S_RZ];
        sc[S_RZ] = rz;
      }
      *cnt = 0u;
    }
  }
}

// iteration count, convergence test, and (Jacobi) beta
__global__ void k_fin_iter(const double* part, int nblk, double* sc, int* done, int jacobi) {
  if (*done) return;
  double rz = block_sum_partials(part, nblk);
  __syncthreads();
  double rr = block_sum_partials(part + nblk, nblk);
  if (threadIdx.x == 0) {
    sc[S_ITS] += 1.0;
    sc[S_RR] = rr;
    if (rr <= sc[S_TOL2] * sc[S_BB]) *done = 1;
    else if (sc[S_ITS] >= sc[S_MAXIT]) *done = 2;
    if (jacobi) {
      sc[S_BETA] = rz / sc[S_RZ];
      sc[S_RZ] = rz;
    }
  }
}

// r.z; with a counter the last block also sets beta = rz_new / rz (first = 1: only rz).
// zf (optional): z as an FP32 multigrid left it, widened into z here
__global__ void k_dot_rz(long long N, const double* r, double* z, double* part, const int* done, double* sc,
                         unsigned* cnt, int first, const float* zf = nullptr) {
  if (*done) return;
  double acc[1] = {0.0};
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < N; id += (long long)gridDim.x * blockDim.x) {
    double zz;
    if (zf) {
      zz = (double)zf[id];
      z[id] = zz;
    } else {
      zz = z[id];
    }
    acc[0] += r[id] * zz;
  }
  block_sum_store<1>(acc, part);
  if (cnt && last_block(cnt)) {
    double rz = block_sum_partials(part, gridDim.x);
    if (threadIdx.x == 0) {
      sc[S_BETA] = first ? 0.0 : rz / sc[S_RZ];
      sc[S_RZ] = rz;
      *cnt = 0u;
    }
  }
}

// beta = rz_new / rz (first == 1: only store rz)
__global__ void k_fin_rz(const double* part, int nblk, double* sc, const int* done, int first) {
  if (*done) return;
  double rz = block_sum_partials(part, nblk);
  if (threadIdx.x == 0) {
    sc[S_BETA] = first ? 0.0 : rz / sc[S_RZ];
    sc[S_RZ] = rz;
  }
}

__global__ void k_p_update(long long N, double* p, const double* z, const double* sc, const int* done) {
  if (*done) return;
  double be = sc[S_BETA];
  const long long gs = (long long)gridDim.x * blockDim.x;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < N; id += 2 * gs) {   // two a trip
    const long long i1 = id + gs < N ? id + gs : id;
    const double z0 = z[id], p0 = p[id], z1 = z[i1], p1 = p[i1];
    p[id] = z0 + be * p0;
    if (i1 != id) p[i1] = z1 + be * p1;
  }
}

// ---------------------------------------------------------------- FP32 defect-correction CG
// Mixed precision for the Helmholtz systems: with the FP64 defect r0 = b - A x0,
// solve A d = r0 by Jacobi-PCG in FP32 (operator, vectors, arithmetic), per-thread
// FP32 partial sums reduced across threads and blocks in FP64, then x = x0 + d in FP64.
struct BoxVf {
  int m[3];
  long long N;
  const float* D;
  const float* c[3];
};

__global__ void k_mx_setup(BoxV A, const double* r64, float* fD, float* fc0, float* fc1, float* fc2, float* fidg,
                           float* fr, float* fz, float* fp, float* fdx, double* part, const int* done, double* sc,
                           unsigned* cnt) {
  if (*done) {   // converged at the initial guess: a zero correction for k_mx_finish
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < A.N; id += (long long)gridDim.x * blockDim.x)
      fdx[id] = 0.f;
    return;
  }
  // the defect scaled by the power of two S_SCL (exact) so that binary32 holds it whatever
  // its size; the convergence test and the statistics then use |b|^2 scaled alike
  const double scl = sc[S_SCL];
  float rz = 0.f;
  float* fc[3] = {fc0, fc1, fc2};
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < A.N; id += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    bdecomp(A.m, id, i, j, k);
    int q[3] = {i, j, k};
    long long st[3] = {1, (long long)A.m[0], (long long)A.m[0] * A.m[1]};
    float D = (float)A.D[id];
    float dt = D;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (!A.c[a]) continue;
      float cl = (float)A.c[a][id];
      fc[a][id] = cl;
      if (q[a] > 0) dt += cl;
      if (q[a] < A.m[a] - 1) dt += (float)A.c[a][id + st[a]];
    }
    fD[id] = D;
    float iv = 1.f / dt;
    fidg[id] = iv;
    float rr = (float)(r64[id] * scl);
    fr[id] = rr;
    float zz = iv * rr;
    fz[id] = zz;
    fp[id] = zz;
    fdx[id] = 0.f;
    rz += rr * zz;
  }
  double acc[1] = {(double)rz};
  block_sum_store<1>(acc, part);
  if (last_block(cnt)) {
    double t = block_sum_partials(part, gridDim.x);
    if (threadIdx.x == 0) {
      sc[S_RZ] = t;
      sc[S_BB] *= scl * scl;
      *cnt = 0u;
    }
  }
}

__global__ void k_spmv_f(BoxVf A, const float* p, float* Ap, double* part, const int* done, double* sc, unsigned* cnt) {
  if (*done) return;
  float acc_f = 0.f;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < A.N; id += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    bdecomp(A.m, id, i, j, k);
    long long st1 = A.m[0], st2 = (long long)A.m[0] * A.m[1];
    float xp = p[id];
    float y = A.D[id] * xp;
    if (i > 0) y += A.c[0][id] * (xp - p[id - 1]);
    if (i < A.m[0] - 1) y += A.c[0][id + 1] * (xp - p[id + 1]);
    if (j > 0) y += A.c[1][id] * (xp - p[id - st1]);
    if (j < A.m[1] - 1) y += A.c[1][id + st1] * (xp - p[id + st1]);
    if (A.c[2]) {
      if (k > 0) y += A.c[2][id] * (xp - p[id - st2]);
      if (k < A.m[2] - 1) y += A.c[2][id + st2] * (xp - p[id + st2]);
    }
    Ap[id] = y;
    acc_f += xp * y;
  }
  double acc[1] = {(double)acc_f};
  block_sum_store<1>(acc, part);
  if (last_block(cnt)) {
    double pap = block_sum_partials(part, gridDim.x);
    if (threadIdx.x == 0) {
      sc[S_PAP] = pap;
      sc[S_ALPHA] = sc[S_RZ] / pap;
      *cnt = 0u;
    }
  }
}

__global__ void k_update_f(long long N, float* dx, float* r, const float* p, const float* Ap, const float* idg, float* z,
                           double* sc, double* part, int* done, unsigned* cnt) {
  if (*done) return;
  float al = (float)sc[S_ALPHA];
  float rz_f = 0.f, rr_f = 0.f;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < N; id += (long long)gridDim.x * blockDim.x) {
    dx[id] += al * p[id];
    float rr = r[id] - al * Ap[id];
    r[id] = rr;
    float zz = idg[id] * rr;
    z[id] = zz;
    rz_f += rr * zz;
    rr_f += rr * rr;
  }
  double acc[2] = {(double)rz_f, (double)rr_f};
  block_sum_store<2>(acc, part);
  if (last_block(cnt)) {
    double rz = block_sum_partials(part, gridDim.x);
    __syncthreads();
    double rr = block_sum_partials(part + gridDim.x, gridDim.x);
    if (threadIdx.x == 0) {
      sc[S_ITS] += 1.0;
      sc[S_RR] = rr;
      if (rr <= sc[S_TOL2] * sc[S_BB]) *done = 1;
      else if (sc[S_ITS] >= sc[S_MAXIT]) *done = 2;
      sc[S_BETA] = rz / sc[S_RZ];
      sc[S_RZ] = rz;
      *cnt = 0u;
    }
  }
}

__global__ void k_p_update_f(long long N, float* p, const float* z, const double* sc, const int* done) {
  if (*done) return;
  float be = (float)sc[S_BETA];
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < N; id += (long long)gridDim.x * blockDim.x)
    p[id] = z[id] + be * p[id];
}

// x = x0 + d (FP64), d the binary32 correction divided by the defect's scale (a power of two)
__global__ void k_mx_finish(long long N, double* x, const float* dx, const double* sc) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id < N) x[id] += (double)dx[id] * sc[S_ISCL];
}

// ---------------------------------------------------------------- persistent Jacobi-PCG
// The whole Jacobi-preconditioned CG of a box system in one cooperative launch.
//
// Form.  Jacobi-PCG on A equals plain CG on the unit-diagonal system
// A^ = S A S, S = diag(A)^(-1/2), with x = S x^ and r^ = S r.  The kernel solves the
// defect equation A d = r0 that way, with r0 normalised to unit length
// (r^0 = S r0 / |r0|), so every working quantity is O(1) and the FP32 variant can
// keep its sums and scalars in FP32 without range trouble.  A^ is applied in matrix
// form, y = x - sum_f c^_f x_nb(f), c^_f = c_f s_P s_nb.  The convergence test is
// the caller's: |r|^2 = |r0|^2 sum_i diag_i r^_i^2 <= rtol^2 |b|^2.
//
// Iteration.  CG in the single-reduction form of Chronopoulos & Gear (1989): with
// w = A^ r^ kept alongside r^, the inner products gamma = r^.r^, delta = w.r^ and the
// weighted residual norm come from one grid-wide sum, after which
//   beta = gamma / gamma_old,  alpha = gamma / (delta - beta gamma / alpha_old),
//   p = r^ + beta p,  s = w + beta s (= A^ p),  x^ += alpha p,  r^ -= alpha s.
// In exact arithmetic the iterates are those of the standard method.  w_new = A^ r^_new
// needs r^_new at the neighbours, which each thread recomputes from the neighbours'
// r^, s, w of the previous iteration; those three vectors are double buffered so no
// cell is overwritten while a neighbour still reads it, and one grid barrier per
// iteration suffices.
//
// Grid sum.  Each block stores its partial sums (buffers alternate with the phase)
// and arrives on a monotone counter; every block waits for the counter to reach
// (phase + 1) x blocks, then warp q adds partial q over all blocks in block order, so
// every block obtains the same totals (deterministic).  One thread forms the scalars
// and broadcasts them through shared memory: GB300 retires about two FP64 FMAs per SM
// clock, so scalar work repeated by every thread is not free.  Waits are bounded:
// past the limit (polls of the arrival counter; a launch argument, so that a caller can
// shorten it) the solve stops (done = 2) and *err is set, so a launch whose blocks were
// not all resident cannot hang; the solve then reports a timeout.
constexpr int PTPB = 512;   // threads per block of the persistent solver
// Boxes from this size on iterate in two passes per CG iteration (the working vectors,
// 13 words a cell, no longer fit in the 129 MB L2)
constexpr long long PERSIST_SPLIT_CELLS = 1LL << 21;



// Grid-wide sums of up to 3 values (nv = 0: a plain barrier) for a cooperative launch
// of PTPB-thread blocks; `phase` counts the grid syncs of the launch (uniform), bar[0]
// the arrivals (zero at launch), `part` holds 2 x NVM x blocks partials.  The totals are
// returned to every thread; false when a wait ran out.  FP32 block sums use warp
// shuffles; FP64 ones go through shared memory so that only three warps do FP64 adds.
template <typename T, int NVM>
__device__ __forceinline__ bool grid_sum(T (&v)[NVM], int nv, int phase, T* part_all, unsigned* bar, int* err,
                                         long long spin_limit) {
  static_assert(NVM <= PTPB / 32, "one warp per value");
  __shared__ T sh[NVM][PTPB / 32];
  __shared__ int ok;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, G = gridDim.x;
  T* part = part_all + (phase & 1) * NVM * G;
  if (nv > 0) {
    if constexpr (sizeof(T) == 8) {
      __shared__ double red[NVM][PTPB];
#pragma unroll
      for (int q = 0; q < NVM; ++q)
        if (q < nv) red[q][threadIdx.x] = v[q];
      __syncthreads();
      if (wid < nv) {
        double t = 0.0;
#pragma unroll
        for (int u = 0; u < PTPB / 32; ++u) t += red[wid][lane + 32 * u];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) part[wid * G + blockIdx.x] = t;
      }
    } else {
#pragma unroll
      for (int q = 0; q < NVM; ++q) {
        if (q >= nv) break;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
        if (lane == 0) sh[q][wid] = v[q];
      }
      __syncthreads();
      if (threadIdx.x < nv) {
        T t = 0;
#pragma unroll
        for (int w = 0; w < PTPB / 32; ++w) t += sh[threadIdx.x][w];
        part[threadIdx.x * G + blockIdx.x] = t;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    volatile unsigned* cnt = bar;
    const unsigned target = (unsigned)(phase + 1) * (unsigned)G;
    long long spins = 0;
    int good = 1;
    while (*cnt < target) {
      if (++spins > spin_limit) { atomicExch(err, 1); good = 0; break; }
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  if (wid < nv) {
    T t = 0;
    for (int b = lane; b < G; b += 32) t += __ldcg(part + wid * G + b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) sh[wid][0] = t;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NVM; ++q)
    if (q < nv) v[q] = sh[q][0];
  const bool r = ok != 0;
  __syncthreads();
  return r;
}

template <typename T>
__device__ __forceinline__ bool grid_sum3(T (&v)[3], int nv, int phase, T* part_all, unsigned* bar, int* err,
                                          long long spin_limit) {
  return grid_sum<T, 3>(v, nv, phase, part_all, bar, err, spin_limit);
}


// End of a persistent solve: statistics (block 0), then the last block to leave
// records whether any wait ran out (stat[S_TMO]; scal_nc[SC_NC] = 2, the step's timeout
// mark, when scal_nc is given) and returns the barrier counters to zero for the next
// launch (no block can still be waiting on them once every block has counted itself out).
__device__ __forceinline__ void persist_finish(double* stat, int* done, const RecordSpec& rec, int its, double rr,
                                               double bb, int result, unsigned* bar, int* err, double* scal_nc) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    stat[S_ITS] = (double)its;
    stat[S_RR] = rr;
    stat[S_BB] = bb;
    const int d = result == 1 ? 1 : 2;
    *done = d;
    if (rec.scal) {
      if (rec.acc) rec.scal[rec.its] += (double)its;
      else rec.scal[rec.its] = (double)its;
      if (rec.res >= 0) rec.scal[rec.res] = bb > 0.0 ? sqrt(rr / bb) : 0.0;
      if (d != 1) rec.scal[SC_NC] = 1.0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned e = atomicAdd(bar + 1, 1u);
    if (e == gridDim.x - 1) {
      __threadfence();
      const int timed_out = atomicAdd(err, 0) != 0;
      stat[S_TMO] = timed_out ? 1.0 : 0.0;
      if (timed_out && scal_nc) scal_nc[SC_NC] = 2.0;
      atomicExch(bar, 0u);
      atomicExch(bar + 1, 0u);
      atomicExch(err, 0);
      __threadfence();
    }
  }
}

template <typename T>
struct PersistArgs {
  BoxV A;                   // FP64 operator (difference form)
  const double* b;          // FP64 right-hand side
  double* x;                // FP64 initial guess in, solution out
  T *ch[3];                 // c^ on the low face of each cell, per axis
  T *dg, *sc;               // diag(A) and S = diag^(-1/2)
  T *r[2], *s[2], *w[2];    // double-buffered r^, s = A^ p, w = A^ r^
  T *p, *dx;                // search direction, x^
  double tol2;              // rtol^2
  int maxit;
  RecordSpec rec;           // statistics slots of this system
};

// Up to three independent systems solved together (the velocity components of the
// momentum predictor are assembled from the same old velocities): each iteration does
// the work of every system still running and one grid-wide sum serves them all, so the
// synchronisation cost of the solves is paid once.  Each system keeps its own
// convergence test, iteration count and statistics.
constexpr int PMAXSYS = 3;
template <typename T>
struct PersistMulti {
  PersistArgs<T> s[PMAXSYS];
  int K;                    // systems
  int split;                // iterate in two passes (large boxes; see the iteration loop)
  T* part;                  // 2 x 3K x blocks partial sums
  double* part64;           // FP64 partials of the initial norms (2 x 2K x blocks)
  double* stat;             // solver scalars (S_*) of the whole solve
  int* done;
  unsigned* bar;            // [0] arrivals, [1] departures (zero at launch)
  int* err;
  long long spin;           // polls of a grid-barrier wait before it gives up
};

template <typename T>
__global__ void __launch_bounds__(PTPB, sizeof(T) == 4 ? 2 : 1) k_pcg_persist(PersistMulti<T> M) {
  // block-uniform state of each system (written by thread 0 between barriers)
  __shared__ double s_bb[PMAXSYS], s_rr[PMAXSYS], s_inv_nu[PMAXSYS];
  __shared__ T s_nu[PMAXSYS], s_thr[PMAXSYS], s_gamma[PMAXSYS], s_alpha[PMAXSYS], s_beta[PMAXSYS], s_rho[PMAXSYS];
  __shared__ int s_its[PMAXSYS], s_res[PMAXSYS], s_act[PMAXSYS], s_any, s_resc[PMAXSYS], s_any_resc;
  const int K = M.K;
  const int gs = gridDim.x * blockDim.x;
  const int id0 = blockIdx.x * blockDim.x + threadIdx.x;
  int phase = 0;
  // phase 0: r0 = b - A x0 in FP64, diag, S = diag^(-1/2); |b|^2 and |r0|^2 per system
  {
    double q64[2 * PMAXSYS];
#pragma unroll
    for (int k = 0; k < 2 * PMAXSYS; ++k) q64[k] = 0.0;
#pragma unroll
    for (int k = 0; k < PMAXSYS; ++k) {
      if (k >= K) break;
      const PersistArgs<T>& a = M.s[k];
      const int N = (int)a.A.N;               // at most PERSIST_MAX_CELLS: 32-bit indices
      for (int id = id0; id < N; id += gs) {
        int i, j, kk;
        bdecomp(a.A.m, id, i, j, kk);
        // the total diagonal, then the defect in the diagonal form d x_P - sum c x_N (one
        // multiply and one FMA per neighbour: fewer binary64 instructions than the difference form)
        const double d = box_diag_total(a.A.m, a.A.D, a.A.c, id, i, j, kk);
        const double ax = box_offdiag(a.A.m, a.A.c, a.x, id, i, j, kk, d * a.x[id]);
        const double bP = a.b[id], r0 = bP - ax;
        a.r[1][id] = (T)r0;                   // rounded once; r[1] is free until the first iteration
        const T dT = (T)d;
        a.dg[id] = dT;
        a.sc[id] = (T)1 / sqrt(dT);
        q64[2 * k] += bP * bP;
        q64[2 * k + 1] += r0 * r0;
      }
    }
    const bool ok = grid_sum<double, 2 * PMAXSYS>(q64, 2 * K, phase++, M.part64, M.bar, M.err, M.spin);
    if (threadIdx.x == 0) {
      s_any = 0;
      s_any_resc = 0;
#pragma unroll
      for (int k = 0; k < PMAXSYS; ++k) {
        s_bb[k] = q64[2 * k];
        s_rr[k] = q64[2 * k + 1];
        s_its[k] = 0;
        s_res[k] = ok ? 2 : 3;
        s_act[k] = 0;
        s_resc[k] = 0;
        if (k < K && ok) {
          if (s_bb[k] == 0.0 || s_rr[k] <= M.s[k].tol2 * s_bb[k]) {
            s_res[k] = 1;                            // converged at the initial guess
          } else {
            // per-solve scalars, formed once (FP64 work repeated by every thread is slow on GB300)
            s_act[k] = 1;
            s_any = 1;
            s_inv_nu[k] = sqrt(s_rr[k]);             // |r0| = 1 / nu
            s_nu[k] = (T)(1.0 / s_inv_nu[k]);
            s_thr[k] = (T)(M.s[k].tol2 * s_bb[k] / s_rr[k]);   // rtol^2 |b|^2 / |r0|^2
            // binary32: a defect of norm outside [2^-100, 2^100] does not survive its
            // rounding to binary32 (entries that matter at the tolerance flush to zero, or
            // nu overflows); it is then formed again and normalised in FP64 before rounding
            if (sizeof(T) == 4 && !(s_inv_nu[k] >= 0x1p-100 && s_inv_nu[k] <= 0x1p100)) {
              s_resc[k] = 1;
              s_any_resc = 1;
            }
          }
        }
      }
    }
    __syncthreads();
  }
  if (s_any_resc) {
    // (a uniform branch: every block holds the same totals) r0 / |r0| in FP64, rounded once
#pragma unroll
    for (int k = 0; k < PMAXSYS; ++k) {
      if (k >= K) break;
      if (!s_resc[k]) continue;
      const PersistArgs<T>& a = M.s[k];
      const int N = (int)a.A.N;
      const double nu64 = 1.0 / s_inv_nu[k];
      for (int id = id0; id < N; id += gs) {
        int i, j, kk;
        bdecomp(a.A.m, id, i, j, kk);
        const double d = box_diag_total(a.A.m, a.A.D, a.A.c, id, i, j, kk);
        const double ax = box_offdiag(a.A.m, a.A.c, a.x, id, i, j, kk, d * a.x[id]);
        a.r[1][id] = (T)((a.b[id] - ax) * nu64);
      }
    }
    double none[1];
    const bool okb = grid_sum<double, 1>(none, 0, phase++, M.part64, M.bar, M.err, M.spin);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < PMAXSYS; ++k) {
        if (k >= K) continue;
        if (s_resc[k]) s_nu[k] = (T)1;           // r[1] holds the normalised defect
        if (!okb && s_act[k]) { s_act[k] = 0; s_res[k] = 3; }   // the barrier wait ran out
      }
      if (!okb) s_any = 0;
    }
    __syncthreads();
  }
  if (s_any) {
    // setup: r^0 = nu S r0 (the neighbours' formed on the fly), c^ on the low faces,
    // w = A^ r^0, s = p = x^ = 0; gamma, delta, weighted |r^|^2
    T v[3 * PMAXSYS];
#pragma unroll
    for (int k = 0; k < 3 * PMAXSYS; ++k) v[k] = 0;
#pragma unroll
    for (int k = 0; k < PMAXSYS; ++k) {
      if (k >= K) break;
      if (!s_act[k]) continue;
      const PersistArgs<T>& a = M.s[k];
      const int m0 = a.A.m[0], m1 = a.A.m[1], m2 = a.A.m[2];
      const int N = (int)a.A.N, st1 = m0, st2 = m0 * m1;
      const bool has2 = a.A.c[2] != nullptr;
      const T nu = s_nu[k];
      const T* r0T = a.r[1];                    // the defect r0 in precision T (phase 0)
      T g = 0, dl = 0, q = 0;
#define RH(o) (nu * a.sc[o] * r0T[o])
      // one cell's r^0, c^ on its low faces, w = A^ r^0 and diagonal (loads and arithmetic only)
      struct SV { T rP, c0, c1, c2, y, d; };
      auto cellv = [&](int id) -> SV {
        int i, j, kk;
        bdecomp(a.A.m, id, i, j, kk);
        SV o;
        const T sP = a.sc[id];
        o.rP = RH(id);
        T y = o.rP;
        o.c0 = 0;
        if (i > 0) {
          o.c0 = (T)a.A.c[0][id] * sP * a.sc[id - 1];
          y -= o.c0 * RH(id - 1);
        }
        if (i < m0 - 1) y -= (T)a.A.c[0][id + 1] * sP * a.sc[id + 1] * RH(id + 1);
        o.c1 = 0;
        if (j > 0) {
          o.c1 = (T)a.A.c[1][id] * sP * a.sc[id - st1];
          y -= o.c1 * RH(id - st1);
        }
        if (j < m1 - 1) y -= (T)a.A.c[1][id + st1] * sP * a.sc[id + st1] * RH(id + st1);
        o.c2 = 0;
        if (has2) {
          if (kk > 0) {
            o.c2 = (T)a.A.c[2][id] * sP * a.sc[id - st2];
            y -= o.c2 * RH(id - st2);
          }
          if (kk < m2 - 1) y -= (T)a.A.c[2][id + st2] * sP * a.sc[id + st2] * RH(id + st2);
        }
        o.y = y;
        o.d = a.dg[id];
        return o;
      };
      auto store = [&](int id, const SV& o) {
        a.r[0][id] = o.rP;
        a.s[0][id] = 0;
        a.p[id] = 0;
        a.dx[id] = 0;
        a.ch[0][id] = o.c0;
        a.ch[1][id] = o.c1;
        if (has2) a.ch[2][id] = o.c2;
        a.w[0][id] = o.y;
        g += o.rP * o.rP;
        dl += o.y * o.rP;
        q += o.d * o.rP * o.rP;
      };
      // two cells a trip (as the iterations' passes): both cells' loads before either's stores
      for (int id = id0; id < N; id += 2 * gs) {
        const int i1 = id + gs < N ? id + gs : id;
        const SV v0 = cellv(id), v1 = cellv(i1);
        store(id, v0);
        if (i1 != id) store(i1, v1);
      }
#undef RH
      v[3 * k] = g;
      v[3 * k + 1] = dl;
      v[3 * k + 2] = q;
    }
    bool ok = grid_sum<T, 3 * PMAXSYS>(v, 3 * K, phase++, M.part, M.bar, M.err, M.spin);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < PMAXSYS; ++k) {
        s_gamma[k] = v[3 * k];
        s_alpha[k] = s_act[k] ? v[3 * k] / v[3 * k + 1] : (T)0;
        s_beta[k] = 0;
        s_rho[k] = v[3 * k + 2];
        if (!ok && s_act[k]) { s_act[k] = 0; s_res[k] = 3; }
      }
    }
    __syncthreads();
    for (int cur = 0;; cur ^= 1) {
      int any = 0;
#pragma unroll
      for (int k = 0; k < PMAXSYS; ++k) any |= (k < K) ? s_act[k] : 0;
      if (!any) break;
#pragma unroll
      for (int k = 0; k < 3 * PMAXSYS; ++k) v[k] = 0;
      bool okA = true;
      if (M.split) {
        // Two passes with a plain grid barrier between them, for boxes far larger than
        // L2: the first updates p, s, x^ and r^ in place, the second forms w = A^ r^ from
        // the stored r^ of the neighbours.  Each pass streams with few loads per cell
        // (the fused form gathers r^, s and w of six neighbours to rebuild their r^);
        // the barrier costs microseconds against a pass of hundreds.  Same arithmetic.
#pragma unroll
        for (int k = 0; k < PMAXSYS; ++k) {
          if (k >= K) break;
          if (!s_act[k]) continue;
          const PersistArgs<T>& a = M.s[k];
          const int N = (int)a.A.N;
          const T al = s_alpha[k], bt = s_beta[k];
          T *r = a.r[0], *s = a.s[0];
          const T* w = a.w[0];
          T g = 0, q = 0;
          // two cells a trip, id and id + gs (the cells and the order of the plain grid-stride
          // loop, so the same sums): the twelve loads of the pair are issued before either
          // cell's stores, twice the loads in flight of one cell per trip
          for (int id = id0; id < N; id += 2 * gs) {
            const int i1 = id + gs < N ? id + gs : id;
            const T rP0 = r[id], p0 = a.p[id], w0 = w[id], s0 = s[id], x0 = a.dx[id], d0 = a.dg[id];
            const T rP1 = r[i1], p1 = a.p[i1], w1 = w[i1], s1 = s[i1], x1 = a.dx[i1], d1 = a.dg[i1];
            {
              const T pP = rP0 + bt * p0;           // p = r^ + beta p
              const T sP = w0 + bt * s0;            // s = w + beta s
              const T rN = rP0 - al * sP;           // r^ -= alpha s
              a.p[id] = pP;
              a.dx[id] = x0 + al * pP;              // x^ += alpha p
              r[id] = rN;
              s[id] = sP;
              g += rN * rN;
              q += d0 * rN * rN;
            }
            if (i1 != id) {
              const T pP = rP1 + bt * p1;
              const T sP = w1 + bt * s1;
              const T rN = rP1 - al * sP;
              a.p[i1] = pP;
              a.dx[i1] = x1 + al * pP;
              r[i1] = rN;
              s[i1] = sP;
              g += rN * rN;
              q += d1 * rN * rN;
            }
          }
          v[3 * k] = g;
          v[3 * k + 2] = q;
        }
        okA = grid_sum<T, 3 * PMAXSYS>(v, 0, phase++, M.part, M.bar, M.err, M.spin);
#pragma unroll
        for (int k = 0; k < PMAXSYS; ++k) {
          if (k >= K) break;
          if (!s_act[k]) continue;
          const PersistArgs<T>& a = M.s[k];
          const int m0 = a.A.m[0], m1 = a.A.m[1], m2 = a.A.m[2];
          const int N = (int)a.A.N, st1 = m0, st2 = m0 * m1;
          const bool has2 = a.A.c[2] != nullptr;
          const T* r = a.r[0];
          T* w = a.w[0];
          T dl = 0;
          // w = A^ r^ of one cell (loads only), with its r^
          auto row = [&](int id, T& rN) -> T {
            int i, j, kk;
            bdecomp(a.A.m, id, i, j, kk);
            rN = r[id];
            const int iw = i > 0 ? id - 1 : id, ie = i < m0 - 1 ? id + 1 : id;
            const int is = j > 0 ? id - st1 : id, in = j < m1 - 1 ? id + st1 : id;
            const T cw = a.ch[0][id], ce = i < m0 - 1 ? a.ch[0][ie] : (T)0;
            const T cs = a.ch[1][id], cn = j < m1 - 1 ? a.ch[1][in] : (T)0;
            T y = rN - (cw * r[iw] + ce * r[ie] + cs * r[is] + cn * r[in]);
            if (has2) {
              const int ib = kk > 0 ? id - st2 : id, it = kk < m2 - 1 ? id + st2 : id;
              const T cb = a.ch[2][id], ct = kk < m2 - 1 ? a.ch[2][it] : (T)0;
              y -= cb * r[ib] + ct * r[it];
            }
            return y;
          };
          // two cells a trip, as in the first pass: both rows are formed before either store
          for (int id = id0; id < N; id += 2 * gs) {
            const int i1 = id + gs < N ? id + gs : id;
            T rN0, rN1;
            const T y0 = row(id, rN0);
            const T y1 = row(i1, rN1);
            w[id] = y0;
            dl += y0 * rN0;
            if (i1 != id) {
              w[i1] = y1;
              dl += y1 * rN1;
            }
          }
          v[3 * k + 1] = dl;
        }
      } else {
#pragma unroll
        for (int k = 0; k < PMAXSYS; ++k) {
          if (k >= K) break;
          if (!s_act[k]) continue;
          const PersistArgs<T>& a = M.s[k];
          const int m0 = a.A.m[0], m1 = a.A.m[1], m2 = a.A.m[2];
          const int N = (int)a.A.N, st1 = m0, st2 = m0 * m1;
          const bool has2 = a.A.c[2] != nullptr;
          const T al = s_alpha[k], bt = s_beta[k];
          const T *r = a.r[cur], *s = a.s[cur], *w = a.w[cur];
          T *rn = a.r[cur ^ 1], *sn = a.s[cur ^ 1], *wn = a.w[cur ^ 1];
          T g = 0, dl = 0, q = 0;
          for (int id = id0; id < N; id += gs) {
            int i, j, kk;
            bdecomp(a.A.m, id, i, j, kk);
            const T rP = r[id];
            const T pP = rP + bt * a.p[id];       // p = r^ + beta p
            const T sP = w[id] + bt * s[id];      // s = w + beta s
            a.p[id] = pP;
            a.dx[id] += al * pP;                  // x^ += alpha p
            const T rN = rP - al * sP;            // r^ -= alpha s
            // neighbours: clamped indices and zero couplings at the box edges, so that all
            // loads issue together; r^_new of a neighbour from its r^, s, w
            const int iw = i > 0 ? id - 1 : id, ie = i < m0 - 1 ? id + 1 : id;
            const int is = j > 0 ? id - st1 : id, in = j < m1 - 1 ? id + st1 : id;
            const T cw = a.ch[0][id], ce = i < m0 - 1 ? a.ch[0][ie] : (T)0;
            const T cs = a.ch[1][id], cn = j < m1 - 1 ? a.ch[1][in] : (T)0;
#define UNB(o) (r[o] - al * (w[o] + bt * s[o]))
            T y = rN - (cw * UNB(iw) + ce * UNB(ie) + cs * UNB(is) + cn * UNB(in));
            if (has2) {
              const int ib = kk > 0 ? id - st2 : id, it = kk < m2 - 1 ? id + st2 : id;
              const T cb = a.ch[2][id], ct = kk < m2 - 1 ? a.ch[2][it] : (T)0;
              y -= cb * UNB(ib) + ct * UNB(it);
            }
#undef UNB
            rn[id] = rN;
            sn[id] = sP;
            wn[id] = y;
            g += rN * rN;
            dl += y * rN;
            q += a.dg[id] * rN * rN;
          }
          v[3 * k] = g;
          v[3 * k + 1] = dl;
          v[3 * k + 2] = q;
        }
      }
      ok = grid_sum<T, 3 * PMAXSYS>(v, 3 * K, phase++, M.part, M.bar, M.err, M.spin) && okA;
      if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < PMAXSYS; ++k) {
          if (k >= K || !s_act[k]) continue;
          ++s_its[k];
          if (!ok) { s_act[k] = 0; s_res[k] = 3; continue; }
          s_rho[k] = v[3 * k + 2];
          if (v[3 * k + 2] <= s_thr[k]) { s_act[k] = 0; s_res[k] = 1; continue; }
          if (s_its[k] >= M.s[k].maxit) { s_act[k] = 0; s_res[k] = 2; continue; }
          const T bn = v[3 * k] / s_gamma[k];
          s_alpha[k] = v[3 * k] / (v[3 * k + 1] - bn * v[3 * k] / s_alpha[k]);
          s_beta[k] = bn;
          s_gamma[k] = v[3 * k];
        }
      }
      __syncthreads();
    }
    // x += S x^ / nu for every system that iterated
#pragma unroll
    for (int k = 0; k < PMAXSYS; ++k) {
      if (k >= K) break;
      if (s_its[k] == 0) continue;
      const PersistArgs<T>& a = M.s[k];
      const int N = (int)a.A.N;
      const double inv_nu = s_inv_nu[k];
      for (int id = id0; id < N; id += 2 * gs) {   // two cells a trip
        const int i1 = id + gs < N ? id + gs : id;
        const double x0 = a.x[id], x1 = a.x[i1];
        const T e0 = a.sc[id] * a.dx[id], e1 = a.sc[i1] * a.dx[i1];
        a.x[id] = x0 + (double)e0 * inv_nu;
        if (i1 != id) a.x[i1] = x1 + (double)e1 * inv_nu;
      }
    }
  }
  // statistics of each system, then of the whole solve, then the barrier reset
  int all = 1, itmax = 0;
  double rrs = 0.0, bbs = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < PMAXSYS; ++k) {
      if (k >= K) break;
      const double rr = s_its[k] > 0 ? (double)s_rho[k] * s_inv_nu[k] * s_inv_nu[k] : s_rr[k];
      const RecordSpec& rec = M.s[k].rec;
      if (blockIdx.x == 0) M.stat[S_ITSK + k] = (double)s_its[k];
      if (blockIdx.x == 0 && rec.scal) {
        if (rec.acc) rec.scal[rec.its] += (double)s_its[k];
        else rec.scal[rec.its] = (double)s_its[k];
        if (rec.res >= 0) rec.scal[rec.res] = s_bb[k] > 0.0 ? sqrt(rr / s_bb[k]) : 0.0;
        if (s_res[k] != 1) rec.scal[SC_NC] = 1.0;
      }
      all = all && s_res[k] == 1;
      itmax = s_its[k] > itmax ? s_its[k] : itmax;
      rrs += rr;
      bbs += s_bb[k];
    }
  }
  const RecordSpec none{nullptr, 0, -1, 0};
  persist_finish(M.stat, M.done, none, itmax, rrs, bbs, all ? 1 : 2, M.bar, M.err, M.s[0].rec.scal);
}



// condition of a solver WHILE node: run another iteration while not done
__global__ void k_set_cond(cudaGraphConditionalHandle h, const int* done) {
  cudaGraphSetConditional(h, *done == 0 ? 1u : 0u);
}

__global__ void k_record(const double* sc, const int* done, double* scal, int slot_its, int slot_res, int accumulate) {
  if (accumulate) scal[slot_its] += sc[S_ITS];
  else scal[slot_its] = sc[S_ITS];
  if (slot_res >= 0) scal[slot_res] = sc[S_BB] > 0.0 ? sqrt(sc[S_RR] / sc[S_BB]) : 0.0;
  if (*done != 1) scal[SC_NC] = 1.0;
}

// ---------------------------------------------------------------- multigrid kernels
template <typename T>
struct LevV {
  int m[3];
  long long N;
  const T* D;
  const T* c[3];
  T* x;
  const T* b;
  const T* idg;
  T* xp;        // post-smoothed iterate of the tiled persistent V-cycle
  // launched V-cycle, levels above its one-block tail (split = 1): 1/diag stored by colour
  // (index col n + t, n = ceil(m0 / 2) m1 m2 cells per colour, t the half sweep's thread of
  // the cell), and bs, b copied into the same layout by each V-cycle's first half sweep, so
  // that a half sweep reads only its own colour's b and 1/diag, whole sectors at a time
  int split;
  T* bs;
};

// one cell of a red-black Gauss-Seidel half sweep: x_P = (b_P + sum c x_nb) / diag_total
// (first = 1: neighbours taken as 0).  Arithmetic in the hierarchy precision T.
// (SPLIT: b and 1/diag read from the colour-ordered copies at ts)
template <typename T, bool SPLIT = false>
__device__ __forceinline__ T gs_value(const LevV<T>& L, long long id, int i, int j, int k, int first,
                                      long long ts = 0) {
  long long st1 = L.m[0], st2 = (long long)L.m[0] * L.m[1];
  T s = SPLIT ? L.bs[ts] : L.b[id];
  if (!first) {
    if (i > 0) s += L.c[0][id] * L.x[id - 1];
    if (i < L.m[0] - 1) s += L.c[0][id + 1] * L.x[id + 1];
    if (j > 0) s += L.c[1][id] * L.x[id - st1];
    if (j < L.m[1] - 1) s += L.c[1][id + st1] * L.x[id + st1];
    if (L.c[2]) {
      if (k > 0) s += L.c[2][id] * L.x[id - st2];
      if (k < L.m[2] - 1) s += L.c[2][id + st2] * L.x[id + st2];
    }
  }
  return s * L.idg[SPLIT ? ts : id];
}

template <typename T, bool SPLIT = false>
__device__ __forceinline__ void gs_cell(const LevV<T>& L, long long id, int i, int j, int k, int first,
                                        long long ts = 0) {
  L.x[id] = gs_value<T, SPLIT>(L, id, i, j, k, first, ts);
}

// One half sweep of colour col over a whole level, one thread per updated cell: thread t
// takes the (t mod h)-th cell of colour col in row t / h (h = ceil(m0 / 2)), so every lane
// of a warp updates a cell.  (A thread per cell with half of them returning issues the
// same binary64 warp instructions for half the work: GB300's FP64 pipe, which retires a
// warp instruction in a fixed number of cycles however many lanes are active, was 91 %
// busy on such a sweep while DRAM ran at 61 %.)
template <typename T, bool SPLIT = false>
__device__ __forceinline__ void grid_half_sweep(const LevV<T>& L, int col, int first, int gid, int gs);

template <typename T, bool SPLIT, int CC>
__device__ __forceinline__ void grid_half_sweep_pair(const LevV<T>& L, int col, int first, int gid, int gs);

// (launched with one thread per CC updated cells)
template <typename T, bool SPLIT, int CC>
__global__ void k_mg_smooth(LevV<T> L, int col, int first, const int* done) {
  if (*done) return;
  grid_half_sweep_pair<T, SPLIT, CC>(L, col, first, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// cells per thread of a launched half sweep: two from this many updated cells on
constexpr long long SWEEP_PAIR_MIN = 1LL << 20;

// threads of a launched half sweep (one per cell of one colour, rows padded to ceil(m0 / 2))
inline long long half_sweep_threads(const int m[3]) { return (long long)((m[0] + 1) >> 1) * m[1] * m[2]; }

// inverse total diagonal of a level
// 1 / (D + sum of adjacent couplings) of one cell, summed in FP64 over the level's values
template <typename T>
__device__ __forceinline__ T mg_idg_cell(const LevV<T>& L, long long id) {
  int i, j, k;
  bdecomp(L.m, id, i, j, k);
  long long st[3] = {1, (long long)L.m[0], (long long)L.m[0] * L.m[1]};
  int q[3] = {i, j, k};
  double dt = (double)L.D[id];
  for (int a = 0; a < 3; ++a) {
    if (!L.c[a] || L.m[a] < 2) continue;
    if (q[a] > 0) dt += (double)L.c[a][id];
    if (q[a] < L.m[a] - 1) dt += (double)L.c[a][id + st[a]];
  }
  return (T)rcp64(dt);   // (the reciprocal by rcp64: within an ulp, no division)
}

template <typename T>
__global__ void k_mg_idg(LevV<T> L, T* idg) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= L.N) return;
  int i, j, k;
  bdecomp(L.m, id, i, j, k);
  long long st[3] = {1, (long long)L.m[0], (long long)L.m[0] * L.m[1]};
  int q[3] = {i, j, k};
  double dt = (double)L.D[id];
  for (int a = 0; a < 3; ++a) {
    if (!L.c[a] || L.m[a] < 2) continue;
    if (q[a] > 0) dt += (double)L.c[a][id];
    if (q[a] < L.m[a] - 1) dt += (double)L.c[a][id + st[a]];
  }
  long long o = id;
  if (L.split) {   // the colour-ordered layout of the launched half sweeps
    const int h = (L.m[0] + 1) >> 1;
    o = (long long)((i + j + k) & 1) * h * L.m[1] * L.m[2] + (long long)(j + L.m[1] * k) * h + (i >> 1);
  }
  idg[o] = (T)rcp64(dt);
}

// residual b - A x of one cell in the hierarchy precision
template <typename T>
__device__ __forceinline__ T mg_resid(const LevV<T>& L, long long id, int i, int j, int k) {
  long long st1 = L.m[0], st2 = (long long)L.m[0] * L.m[1];
  T xp = L.x[id];
  T y = L.D[id] * xp;
  if (i > 0) y += L.c[0][id] * (xp - L.x[id - 1]);
  if (i < L.m[0] - 1) y += L.c[0][id + 1] * (xp - L.x[id + 1]);
  if (j > 0) y += L.c[1][id] * (xp - L.x[id - st1]);
  if (j < L.m[1] - 1) y += L.c[1][id + st1] * (xp - L.x[id + st1]);
  if (L.c[2]) {
    if (k > 0) y += L.c[2][id] * (xp - L.x[id - st2]);
    if (k < L.m[2] - 1) y += L.c[2][id + st2] * (xp - L.x[id + st2]);
  }
  return L.b[id] - y;
}

// the residual with the level's total diagonal a_P = D + sum c given: b - a_P x_P + sum c x_N
// (one FMA per term: the diagonal form of the FP64 CG operator, for level 0 of an FP64
// hierarchy, whose total diagonal the CG's set-up has formed)
__device__ __forceinline__ double mg_resid_diag(const LevV<double>& L, const double* ad, long long id, int i, int j,
                                                int k) {
  const long long st1 = L.m[0], st2 = (long long)L.m[0] * L.m[1];
  double r = fma(-ad[id], L.x[id], L.b[id]);
  if (i > 0) r = fma(L.c[0][id], L.x[id - 1], r);
  if (i < L.m[0] - 1) r = fma(L.c[0][id + 1], L.x[id + 1], r);
  if (j > 0) r = fma(L.c[1][id], L.x[id - st1], r);
  if (j < L.m[1] - 1) r = fma(L.c[1][id + st1], L.x[id + st1], r);
  if (L.c[2]) {
    if (k > 0) r = fma(L.c[2][id], L.x[id - st2], r);
    if (k < L.m[2] - 1) r = fma(L.c[2][id + st2], L.x[id + st2], r);
  }
  return r;
}

// residual of the fine level restricted (summed) into the coarse right-hand side; ad (FP64
// levels only, may be null): the fine level's total diagonal, for the diagonal form
template <typename T>
__global__ void k_mg_restrict(LevV<T> F, LevV<T> C, const int* done, const T* ad = nullptr) {
  if (*done) return;
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= C.N) return;
  int I, J, K;
  bdecomp(C.m, id, I, J, K);
  int kz = F.m[2] > 1 ? 2 : 1;
  T s = 0;
  for (int dk = 0; dk < kz; ++dk)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        int i = 2 * I + di, j = 2 * J + dj, k = kz == 2 ? 2 * K + dk : 0;
        long long fi = (long long)i + (long long)F.m[0] * ((long long)j + (long long)F.m[1] * k);
        if constexpr (sizeof(T) == 8) {
          if (ad) {
            s += mg_resid_diag(F, ad, fi, i, j, k);
            continue;
          }
        }
        s += mg_resid<T>(F, fi, i, j, k);
      }
  ((T*)C.b)[id] = s;
}

template <typename T>
__global__ void k_mg_prolong(LevV<T> F, LevV<T> C, const int* done) {
  if (*done) return;
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= F.N) return;
  int i, j, k;
  bdecomp(F.m, id, i, j, k);
  int K = F.m[2] > 1 ? k / 2 : 0;
  long long ci = (long long)(i / 2) + (long long)C.m[0] * ((long long)(j / 2) + (long long)C.m[1] * K);
  F.x[id] = F.x[id] + C.x[ci];
}

// coarse operator: couplings = 1/2 sum of the fine couplings across the coarse face, D = 1/2 sum
template <typename T>
__device__ __forceinline__ void mg_coarsen_cell(const LevV<T>& F, const LevV<T>& C, long long id, T* Dc, T* c0, T* c1,
                                                T* c2);

template <typename T>
__global__ void k_mg_coarsen(LevV<T> F, LevV<T> C, T* Dc, T* c0, T* c1, T* c2) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= C.N) return;
  mg_coarsen_cell<T>(F, C, id, Dc, c0, c1, c2);
}

template <typename T>
__device__ __forceinline__ void mg_coarsen_cell(const LevV<T>& F, const LevV<T>& C, long long id, T* Dc, T* c0, T* c1,
                                                T* c2) {
  int I, J, K;
  bdecomp(C.m, id, I, J, K);
  int kz = F.m[2] > 1 ? 2 : 1;
  double d = 0.0, s[3] = {0, 0, 0};
  T* cc[3] = {c0, c1, c2};
  for (int dk = 0; dk < kz; ++dk)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        int i = 2 * I + di, j = 2 * J + dj, k = kz == 2 ? 2 * K + dk : 0;
        long long fi = (long long)i + (long long)F.m[0] * ((long long)j + (long long)F.m[1] * k);
        d += (double)F.D[fi];
        if (di == 0) s[0] += (double)F.c[0][fi];
        if (dj == 0) s[1] += (double)F.c[1][fi];
        if (kz == 2 && dk == 0) s[2] += (double)F.c[2][fi];
      }
  Dc[id] = (T)(0.5 * d);
  for (int a = 0; a < 3; ++a)
    if (cc[a]) cc[a][id] = (T)(0.5 * s[a]);
}

// V-cycle of levels l0 .. nl-1 inside one thread block (small levels: one launch
// instead of ten per level).  Same operations and order as the per-level kernels.
// The iterate x of every tail level and the right-hand side b of the levels the tail
// restricts to live in shared memory (the sweeps would otherwise wait on L2 after
// every half sweep); the operator and the first tail level's b are read through L1.
constexpr int TAIL_MAX_CELLS = 8192;
constexpr int TAIL_THREADS = 1024;
template <typename T>
struct TailLevels {
  LevV<T> L[24];
  int xo[24], bo[24];   // shared-memory offsets (elements) of x and b per level
  int total;            // shared-memory elements
};

// shared-memory elements of a tail over levels of sizes N[l0..nl-1]: x of every level,
// b of every level but the first, each rounded up to 16 bytes
static long long tail_layout(const MGLevel* lev, int l0, int nl, size_t es, int* xo, int* bo) {
  const long long al = 16 / (long long)es;
  long long off = 0;
  for (int l = l0; l < nl; ++l) {
    if (xo) xo[l] = (int)off;
    off += (lev[l].N + al - 1) / al * al;
  }
  for (int l = l0 + 1; l < nl; ++l) {
    if (bo) bo[l] = (int)off;
    off += (lev[l].N + al - 1) / al * al;
  }
  return off;
}

// one red-black half sweep over the cells of colour `col` only (half rows)
// the threads that run the tail: the whole block
struct TailBlock {
  __device__ static int tid() { return threadIdx.x; }
  __device__ static int n() { return blockDim.x; }
  __device__ static void sync() { __syncthreads(); }
};

// one red-black half sweep over the cells of colour `col` only (half rows)
template <typename T, class G = TailBlock>
__device__ void tail_smooth(const LevV<T>& L, int col, int first) {
  const int m0 = L.m[0], m1 = L.m[1], h = (m0 + 1) >> 1;
  const int n = h * m1 * L.m[2];
  for (int t = G::tid(); t < n; t += G::n()) {
    const int row = t / h, q = t - row * h;
    const int k = row / m1, j = row - k * m1;
    const int i = 2 * q + ((j + k + col) & 1);
    if (i < m0) gs_cell<T>(L, (long long)i + (long long)m0 * row, i, j, k, first);
  }
  G::sync();
}

// pre-smoothing of F and the restriction of its residual into C.b
template <typename T, class G>
__device__ void tail_down(const LevV<T>& F, const LevV<T>& C, int nu) {
  for (int s = 0; s < nu; ++s) {
    tail_smooth<T, G>(F, 0, s == 0);
    tail_smooth<T, G>(F, 1, 0);
  }
  const int kz = F.m[2] > 1 ? 2 : 1;
  for (long long id = G::tid(); id < C.N; id += G::n()) {
    int I, J, K;
    bdecomp(C.m, id, I, J, K);
    T s = 0;
    for (int dk = 0; dk < kz; ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
          int i = 2 * I + di, j = 2 * J + dj, k = kz == 2 ? 2 * K + dk : 0;
          long long fi = (long long)i + (long long)F.m[0] * ((long long)j + (long long)F.m[1] * k);
          s += mg_resid<T>(F, fi, i, j, k);
        }
    ((T*)C.b)[id] = s;
  }
  G::sync();
}

// the coarsest level: ncoarse symmetric sweep pairs
template <typename T, class G>
__device__ void tail_coarsest(const LevV<T>& L, int ncoarse) {
  for (int s = 0; s < ncoarse; ++s) {
    tail_smooth<T, G>(L, 0, s == 0);
    tail_smooth<T, G>(L, 1, 0);
  }
  for (int s = 0; s < ncoarse; ++s) {
    tail_smooth<T, G>(L, 1, 0);
    tail_smooth<T, G>(L, 0, 0);
  }
}

// prolongation F.x += C.x and post-smoothing of F
template <typename T, class G>
__device__ void tail_up(const LevV<T>& F, const LevV<T>& C, int nu) {
  for (long long id = G::tid(); id < F.N; id += G::n()) {
    int i, j, k;
    bdecomp(F.m, id, i, j, k);
    int K = F.m[2] > 1 ? k / 2 : 0;
    long long ci = (long long)(i / 2) + (long long)C.m[0] * ((long long)(j / 2) + (long long)C.m[1] * K);
    F.x[id] = F.x[id] + C.x[ci];
  }
  G::sync();
  for (int s = 0; s < nu; ++s) {
    tail_smooth<T, G>(F, 1, 0);
    tail_smooth<T, G>(F, 0, 0);
  }
}

// ---------------------------------------------------------------- dense coarsest level
// The coarsest level of the persistent V-cycle (at most DENSE_MAX_CELLS cells) is solved
// exactly instead of by red-black sweeps: its operator A (SPD: diagonal D + adjacent
// couplings, off-diagonals -c) is factored once per solve by Gaussian elimination
// without pivoting on [A | I].  Elimination turns A into U = diag(d) L^T and I into
// E = L^-1 (A = L diag(d) L^T, L unit lower triangular), so A^-1 = W^T W with
// W = diag(d)^-1/2 E.  Applying x = W^T (W b) is two dense triangular products -- a
// handful of block-wide steps where the sweeps took dozens -- and keeps the coarse
// solve symmetric positive definite, as the CG preconditioner requires.
constexpr int DENSE_MAX_CELLS = 64;
constexpr int DENSE_GROUPS = PTPB / DENSE_MAX_CELLS;   // row groups of the factorisation
static_assert(DENSE_GROUPS >= 1, "one thread per (column, row group)");

// shared-memory elements of the dense coarse solve: W (n x (n + 1)) and y = W b
__host__ __device__ constexpr int dense_elems(int n) {
  return n > 0 ? n * (n + 1) + DENSE_MAX_CELLS : 0;
}

// Factor the operator of level L (n cells) into W at `W` (row stride n + 1), using
// `A` (n x n) as scratch.  Called by a whole block of at least DENSE_GROUPS x
// DENSE_MAX_CELLS threads (PTPB).  Returns (to every thread) whether all pivots were positive
// and finite; otherwise W must not be used.
template <typename T>
__device__ bool dense_factor(const LevV<T>& L, int n, T* W, T* A) {
  const int ws = n + 1;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    A[e] = T(0);
    const int r = e / n, c = e - r * n;
    W[r * ws + c] = r == c ? T(1) : T(0);
  }
  __syncthreads();
  for (int id = threadIdx.x; id < n; id += blockDim.x) {
    int q[3];
    bdecomp(L.m, id, q[0], q[1], q[2]);
    const int st[3] = {1, L.m[0], L.m[0] * L.m[1]};
    double dt = (double)L.D[id];
    for (int a = 0; a < 3; ++a) {
      if (!L.c[a] || L.m[a] < 2) continue;
      if (q[a] > 0) {
        dt += (double)L.c[a][id];
        A[id * n + id - st[a]] = -L.c[a][id];
      }
      if (q[a] < L.m[a] - 1) {
        dt += (double)L.c[a][id + st[a]];
        A[id * n + id + st[a]] = -L.c[a][id + st[a]];
      }
    }
    A[id * n + id] = (T)dt;
  }
  __syncthreads();
  // step k: rows i > k of the lower triangle, A_ij -= (A_ik / A_kk) A_jk for k < j <= i
  // (the trailing matrix stays symmetric), and E_ij -= (A_ik / A_kk) E_kj for j <= k.
  // Thread (g, j): column j, rows k + 1 + g, k + 1 + g + DENSE_GROUPS, ..., taken
  // DENSE_UNROLL at a time with all loads ahead of the stores (column k and row k of E,
  // which the step reads, are not written by it).
  constexpr int DENSE_UNROLL = 8;
  const int j = threadIdx.x % DENSE_MAX_CELLS, g = threadIdx.x / DENSE_MAX_CELLS;
  const bool act = g < DENSE_GROUPS && j < n;
  for (int k = 0; k < n; ++k) {
    if (act) {
      const T rp = T(1) / A[k * n + k];
      const bool upd_a = j > k;
      const T m = upd_a ? A[j * n + k] * rp : W[k * ws + j] * rp;
      T* col = upd_a ? A + j : W + j;
      const int cs = upd_a ? n : ws;
      for (int i0 = k + 1 + g; i0 < n; i0 += DENSE_GROUPS * DENSE_UNROLL) {
        T f[DENSE_UNROLL], v[DENSE_UNROLL];
#pragma unroll
        for (int u = 0; u < DENSE_UNROLL; ++u) {
          const int i = i0 + u * DENSE_GROUPS;
          const bool in = i < n && (!upd_a || j <= i);
          f[u] = in ? A[i * n + k] : T(0);
          v[u] = in ? col[i * cs] : T(0);
        }
#pragma unroll
        for (int u = 0; u < DENSE_UNROLL; ++u) {
          const int i = i0 + u * DENSE_GROUPS;
          if (i < n && (!upd_a || j <= i)) col[i * cs] = v[u] - f[u] * m;
        }
      }
    }
    __syncthreads();
  }
  // W = diag(d)^-1/2 E with the pivots d_k = A_kk (their scales in A's first column,
  // which nothing reads any more)
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const T d = A[r * n + r];
    if (!(d > T(0)) || !(d < T(1e30))) bad = 1;
    A[r * n] = T(1) / sqrt(d);
  }
  __syncthreads();
  if (act)
    for (int r = j + g; r < n; r += DENSE_GROUPS) W[r * ws + j] *= A[r * n];
  __syncthreads();
  return bad == 0;
}

// x = W^T (W b) on n <= DENSE_MAX_CELLS cells by the calling block, y = W b held in
// P.  One thread per cell and product; consecutive threads take consecutive cells, so
// the padded row stride n + 1 keeps both products free of bank conflicts.
template <typename T, class G>
__device__ void dense_apply(const T* W, int n, T* P, const T* b, T* x) {
  const int ws = n + 1;
  for (int c = G::tid(); c < n; c += G::n()) {   // y_c = sum_{i <= c} W_ci b_i
    T s = T(0);
#pragma unroll 4
    for (int i = 0; i <= c; ++i) s += W[c * ws + i] * b[i];
    P[c] = s;
  }
  G::sync();
  for (int c = G::tid(); c < n; c += G::n()) {   // x_c = sum_{r >= c} W_rc y_r
    T s = T(0);
#pragma unroll 4
    for (int r = c; r < n; ++r) s += W[r * ws + c] * P[r];
    x[c] = s;
  }
  G::sync();
}

// the dense coarsest level of a tail: W and y in shared memory (n = 0: none, the
// coarsest level is swept)
template <typename T>
struct DenseCoarse {
  const T* W;
  T* P;
  int n;
};

template <typename T>
__device__ __forceinline__ LevV<T> tail_level(const TailLevels<T>& TL, T* sm, int l, int l0) {
  LevV<T> L = TL.L[l];
  L.x = sm + TL.xo[l];
  if (l > l0) L.b = sm + TL.bo[l];
  return L;
}

// V-cycle of the tail levels l0 .. nl-1 by the calling block; x and the restricted b
// in shared memory `sm` (layout TL.xo / TL.bo); level l0's b is read from global
// memory and its x written back there at the end.
template <typename T>
__device__ void tail_vcycle(const TailLevels<T>& TL, T* sm, int l0, int nl, int nu, int ncoarse,
                            const DenseCoarse<T>& dc = DenseCoarse<T>{nullptr, nullptr, 0}) {
  for (int l = l0; l < nl - 1; ++l)
    tail_down<T, TailBlock>(tail_level<T>(TL, sm, l, l0), tail_level<T>(TL, sm, l + 1, l0), nu);
  {
    const LevV<T> Lc = tail_level<T>(TL, sm, nl - 1, l0);
    if (dc.n > 0) dense_apply<T, TailBlock>(dc.W, dc.n, dc.P, Lc.b, Lc.x);
    else tail_coarsest<T, TailBlock>(Lc, ncoarse);
  }
  for (int l = nl - 2; l >= l0; --l)
    tail_up<T, TailBlock>(tail_level<T>(TL, sm, l, l0), tail_level<T>(TL, sm, l + 1, l0), nu);
  // the first tail level's x goes back to global memory for the prolongation above
  const T* xs = sm + TL.xo[l0];
  for (long long id = threadIdx.x; id < TL.L[l0].N; id += blockDim.x) TL.L[l0].x[id] = xs[id];
}

template <typename T>
__global__ void __launch_bounds__(TAIL_THREADS) k_mg_tail(TailLevels<T> TL, int l0, int nl, int nu, int ncoarse,
                                                          const int* done) {
  if (*done) return;
  extern __shared__ __align__(16) unsigned char tail_smem[];
  tail_vcycle<T>(TL, reinterpret_cast<T*>(tail_smem), l0, nl, nu, ncoarse);
}

// ---------------------------------------------------------------- persistent MG-PCG
// The whole multigrid-preconditioned CG of the pressure system in one cooperative
// launch (single droplets of a latency-bound size).  The preconditioner is the V-cycle
// of the launched path, operation for operation (same sweeps, order, transfer and
// precision), so the iterates agree with it up to the order of the inner-product sums.
//
// Outer iteration: CG in the single-reduction form of Chronopoulos & Gear with the
// preconditioner, in FP64: z = M r, w = A z, gamma = r.z and delta = w.z from one grid
// sum, then beta = gamma / gamma_old, alpha = gamma / (delta - beta gamma / alpha_old),
// p = z + beta p, q = w + beta q (= A p), x += alpha p, r -= alpha q.  The update is
// fused with the start of the next V-cycle (r cast into the level-0 right-hand side
// and the first red half sweep, x = b / diag), and |r|^2 travels with that phase's
// barrier, so the convergence test sees each new residual before any further work.
//
// V-cycle phases, each ended by a grid barrier: half sweeps over the cells of one
// colour; the restriction fused with the coarse level's first red half sweep (which
// needs only the cell's own b); the prolongation fused with the fine level's first
// black half sweep, whose red neighbours take their corrected value x + x_coarse on
// the fly (the red cells' own corrected values are read by nothing else: the next red
// half sweep overwrites them from their black neighbours).  Levels of at most
// PMG_TAIL_MAX_CELLS cells run in block 0 out of shared memory while the other blocks
// wait at the barrier.
constexpr int PMG_TAIL_MAX_CELLS = 2048;

// half sweep of colour `col` over a whole level, grid-strided
template <typename T, bool SPLIT>
__device__ __forceinline__ void grid_half_sweep(const LevV<T>& L, int col, int first, int gid, int gs) {
  const int m0 = L.m[0], m1 = L.m[1], h = (m0 + 1) >> 1;
  const int n = h * m1 * L.m[2];
  for (int t = gid; t < n; t += gs) {
    const int row = t / h, q = t - row * h;
    const int k = row / m1, j = row - k * m1;
    const int i = 2 * q + ((j + k + col) & 1);
    if (SPLIT && first) {
      // the V-cycle's first (red) half sweep of the level: both cells of this thread's pair
      // copy their b into the colour-ordered layout (whole sectors read) for the later sweeps
      const int ib = 2 * q + ((j + k + 1) & 1);
      if (i < m0) L.bs[t] = L.b[(long long)i + (long long)m0 * row];
      if (ib < m0) L.bs[(long long)n + t] = L.b[(long long)ib + (long long)m0 * row];
    }
    if (i < m0) gs_cell<T, SPLIT>(L, (long long)i + (long long)m0 * row, i, j, k, first, (long long)col * n + t);
  }
}

// The same half sweep with CC cells per thread and trip (t, t + gs, ...): all the cells'
// loads are issued before any store (cells of one colour are never neighbours, so the values
// are those of separate updates).  On a large level a launched half sweep at one cell per
// thread keeps too few loads in flight per SM to cover the latency of its gathers; two cells
// a thread run faster there (four were slower: fewer threads, more registers), while small
// levels, with a wave of threads or less, lose more to the longer thread than they gain.
template <typename T, bool SPLIT, int CC>
__device__ __forceinline__ void grid_half_sweep_pair(const LevV<T>& L, int col, int first, int gid, int gs) {
  constexpr int SWEEP_CELLS = CC;
  const int m0 = L.m[0], m1 = L.m[1], h = (m0 + 1) >> 1;
  const int n = h * m1 * L.m[2];
  for (int t0 = gid; t0 < n; t0 += SWEEP_CELLS * gs) {
    T v[SWEEP_CELLS];
    long long at[SWEEP_CELLS];
#pragma unroll
    for (int u = 0; u < SWEEP_CELLS; ++u) at[u] = -1;
#pragma unroll
    for (int u = 0; u < SWEEP_CELLS; ++u) {
      const int t = t0 + u * gs;
      if (t >= n) break;
      const int row = t / h, q = t - row * h;
      const int k = row / m1, j = row - k * m1;
      const int i = 2 * q + ((j + k + col) & 1);
      if (SPLIT && first) {   // (as in grid_half_sweep)
        const int ib = 2 * q + ((j + k + 1) & 1);
        if (i < m0) L.bs[t] = L.b[(long long)i + (long long)m0 * row];
        if (ib < m0) L.bs[(long long)n + t] = L.b[(long long)ib + (long long)m0 * row];
      }
      if (i < m0) {
        at[u] = (long long)i + (long long)m0 * row;
        v[u] = gs_value<T, SPLIT>(L, at[u], i, j, k, first, (long long)col * n + t);
      }
    }
#pragma unroll
    for (int u = 0; u < SWEEP_CELLS; ++u)
      if (at[u] >= 0) L.x[at[u]] = v[u];
  }
}

// C.b = restricted residual of F; with `red`, also the first (red) half sweep on C
template <typename T>
__device__ __forceinline__ void grid_restrict(const LevV<T>& F, const LevV<T>& C, bool red, int gid, int gs) {
  const int kz = F.m[2] > 1 ? 2 : 1;
  for (long long id = gid; id < C.N; id += gs) {
    int I, J, K;
    bdecomp(C.m, id, I, J, K);
    T s = 0;
    for (int dk = 0; dk < kz; ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
          int i = 2 * I + di, j = 2 * J + dj, k = kz == 2 ? 2 * K + dk : 0;
          long long fi = (long long)i + (long long)F.m[0] * ((long long)j + (long long)F.m[1] * k);
          s += mg_resid<T>(F, fi, i, j, k);
        }
    ((T*)C.b)[id] = s;
    if (red && ((I + J + K) & 1) == 0) C.x[id] = s * C.idg[id];
  }
}

// x of F at a cell plus its coarse-level correction
template <typename T>
__device__ __forceinline__ T prolonged(const LevV<T>& F, const LevV<T>& C, const T* cx, long long id, int i, int j,
                                      int k) {
  const int K = F.m[2] > 1 ? k / 2 : 0;
  const long long ci = (long long)(i / 2) + (long long)C.m[0] * ((long long)(j / 2) + (long long)C.m[1] * K);
  return F.x[id] + cx[ci];
}

// prolongation F.x += C.x fused with the black half sweep of F (same arithmetic as
// the separate prolongation followed by gs_cell)
template <typename T>
__device__ __forceinline__ void grid_prolong_black(const LevV<T>& F, const LevV<T>& C, int gid, int gs) {
  const int m0 = F.m[0], m1 = F.m[1], m2 = F.m[2], h = (m0 + 1) >> 1;
  const int n = h * m1 * m2;
  const long long st1 = m0, st2 = (long long)m0 * m1;
  for (int t = gid; t < n; t += gs) {
    const int row = t / h, q = t - row * h;
    const int k = row / m1, j = row - k * m1;
    const int i = 2 * q + ((j + k + 1) & 1);
    if (i >= m0) continue;
    const long long id = (long long)i + (long long)m0 * row;
    T s = F.b[id];
    if (i > 0) s += F.c[0][id] * prolonged<T>(F, C, C.x, id - 1, i - 1, j, k);
    if (i < m0 - 1) s += F.c[0][id + 1] * prolonged<T>(F, C, C.x, id + 1, i + 1, j, k);
    if (j > 0) s += F.c[1][id] * prolonged<T>(F, C, C.x, id - st1, i, j - 1, k);
    if (j < m1 - 1) s += F.c[1][id + st1] * prolonged<T>(F, C, C.x, id + st1, i, j + 1, k);
    if (F.c[2]) {
      if (k > 0) s += F.c[2][id] * prolonged<T>(F, C, C.x, id - st2, i, j, k - 1);
      if (k < m2 - 1) s += F.c[2][id + st2] * prolonged<T>(F, C, C.x, id + st2, i, j, k + 1);
    }
    F.x[id] = s * F.idg[id];
  }
}

// The launched V-cycle's prolongation x_F += x_C fused with the first post-smoothing half
// sweep (colour 1) of F, for binary32 levels.  A colour-1 cell's update reads only its
// colour-0 neighbours, each taken as x_F + x_C of its parent (the prolonged value, rounded
// as the separate prolongation rounds it), and overwrites the cell's own x; the colour-0
// cells' prolonged values are read by nothing else, as the colour-0 half sweep that
// follows overwrites them from their colour-1 neighbours.  So the level ends with the
// values of the prolongation followed by the half sweep, with one pass over the level
// fewer.  (A binary64 level keeps the separate pass: six additions per updated cell in
// place of the prolongation's one per cell weigh on GB300's binary64 pipe.)
// (CC cells a thread and trip, as the launched half sweeps)
template <typename T, bool SPLIT, int CC>
__global__ void k_mg_prolong_smooth(LevV<T> F, LevV<T> C, const int* done) {
  constexpr int SWEEP_CELLS = CC;
  if (*done) return;
  const int m0 = F.m[0], m1 = F.m[1], m2 = F.m[2], h = (m0 + 1) >> 1;
  const int n = h * m1 * m2;
  const long long st1 = m0, st2 = (long long)m0 * m1;
  const int gs = gridDim.x * blockDim.x;
  for (int t0 = blockIdx.x * blockDim.x + threadIdx.x; t0 < n; t0 += SWEEP_CELLS * gs) {
    T v[SWEEP_CELLS];
    long long at[SWEEP_CELLS];
#pragma unroll
    for (int u = 0; u < SWEEP_CELLS; ++u) at[u] = -1;
#pragma unroll
    for (int u = 0; u < SWEEP_CELLS; ++u) {
      const int t = t0 + u * gs;
      if (t >= n) break;
      const int row = t / h, q = t - row * h;
      const int k = row / m1, j = row - k * m1;
      const int i = 2 * q + ((j + k + 1) & 1);
      if (i >= m0) continue;
      const long long id = (long long)i + (long long)m0 * row, ts = (long long)n + t;
      T s = SPLIT ? F.bs[ts] : F.b[id];
      if (i > 0) s += F.c[0][id] * prolonged<T>(F, C, C.x, id - 1, i - 1, j, k);
      if (i < m0 - 1) s += F.c[0][id + 1] * prolonged<T>(F, C, C.x, id + 1, i + 1, j, k);
      if (j > 0) s += F.c[1][id] * prolonged<T>(F, C, C.x, id - st1, i, j - 1, k);
      if (j < m1 - 1) s += F.c[1][id + st1] * prolonged<T>(F, C, C.x, id + st1, i, j + 1, k);
      if (F.c[2]) {
        if (k > 0) s += F.c[2][id] * prolonged<T>(F, C, C.x, id - st2, i, j, k - 1);
        if (k < m2 - 1) s += F.c[2][id + st2] * prolonged<T>(F, C, C.x, id + st2, i, j, k + 1);
      }
      at[u] = id;
      v[u] = s * F.idg[SPLIT ? ts : id];
    }
#pragma unroll
    for (int u = 0; u < SWEEP_CELLS; ++u)
      if (at[u] >= 0) F.x[at[u]] = v[u];
  }
}

// Temporal blocking of the smoothing on 2D levels: each block takes a tx x ty tile,
// loads it with THALO rings into shared memory and runs all 2 nu half sweeps there.
// Half sweep s updates the cells within THALO - s rings of the tile (clipped to the
// level), which read only cells updated by half sweep s - 1, so the tile's cells end
// with exactly the values of the level-wide sweeps (same arithmetic, same order) and a
// whole pre- or post-smoothing costs one grid barrier instead of 2 nu.  One ring more
// than the half sweeps need leaves the owned cells' neighbours exact too, so the
// pre-smoothing phase also forms the owned cells' residuals and restricts them into
// the coarse right-hand side (tiles are even, so 2 x 2 aggregates never straddle two).
constexpr int MG_NU = 2;                       // red-black sweeps before and after
constexpr int THALO = 2 * MG_NU + 1;           // rings: one per half sweep, plus one

// cells of the region of a tx x ty tile (the tile shape is a launch parameter, chosen
// by the autotuner)
__host__ __device__ constexpr int tile_region(int tx, int ty) { return (tx + 2 * THALO) * (ty + 2 * THALO); }
constexpr int TILE_ARRAYS = 6;                 // x, b, 1 / diag, c0, c1, D

// dynamic shared memory of the persistent MG-PCG (elements): the tail, then the
// TILE_ARRAYS tile arrays (the dense factorisation's scratch matrix while it runs,
// before the first V-cycle), then W and y of a dense coarsest level of dn cells
struct PmgLayout {
  int tiles, dw, dp;
  size_t bytes;
};
static PmgLayout pmg_layout(int tail_elems, size_t es, int tx, int ty, int dn) {
  PmgLayout L;
  L.tiles = (tail_elems + 3) / 4 * 4;
  L.dw = L.tiles + std::max(TILE_ARRAYS * tile_region(tx, ty), dn * dn);
  L.dp = L.dw + dn * (dn + 1);
  L.bytes = (size_t)(L.dw + dense_elems(dn)) * es;
  return L;
}

// the level solved densely by the persistent V-cycle of an FP32 hierarchy: the first
// tail level (from lt on) of at most DENSE_MAX_CELLS cells, or -1 (coarsest level swept)
static int dense_level(const MGLevel* lev, int lt, int nlev, bool f32) {
  if (!f32) return -1;
  for (int l = lt; l < nlev; ++l)
    if (lev[l].N <= DENSE_MAX_CELLS) return l;
  return -1;
}

template <typename T>
struct TileSmem {
  T *x, *b, *idg, *c0, *c1, *D;
};

struct TileBox {
  int oi0, oi1, oj0, oj1;   // owned cells
  int i0, j0, rx, ry;       // region origin and extent (owned + THALO rings, clipped)
};

__device__ __forceinline__ TileBox tile_box(int m0, int m1, int t, int TX, int TY) {
  const int ntx = (m0 + TX - 1) / TX;
  const int ty = t / ntx, tx = t - ty * ntx;
  TileBox B;
  B.oi0 = tx * TX;
  B.oi1 = min(B.oi0 + TX, m0);
  B.oj0 = ty * TY;
  B.oj1 = min(B.oj0 + TY, m1);
  B.i0 = max(B.oi0 - THALO, 0);
  B.j0 = max(B.oj0 - THALO, 0);
  B.rx = min(B.oi1 + THALO, m0) - B.i0;
  B.ry = min(B.oj1 + THALO, m1) - B.j0;
  return B;
}

__device__ __forceinline__ int tile_count(int m0, int m1, int TX, int TY) {
  return ((m0 + TX - 1) / TX) * ((m1 + TY - 1) / TY);
}

// the 2 nu half sweeps of a loaded tile; pre: red (from b alone), black, red, black;
// post: black, red, black, red (gs_cell's arithmetic)
template <typename T>
__device__ void tile_sweeps(const TileSmem<T>& S, const TileBox& B, int m0, int m1, bool pre) {
  for (int s = 1; s <= 2 * MG_NU; ++s) {
    const int col = pre ? ((s - 1) & 1) : (s & 1);
    const int ring = THALO - s;
    const int a0 = max(B.oi0 - ring, 0), a1 = min(B.oi1 + ring, m0);
    const int b0 = max(B.oj0 - ring, 0), b1 = min(B.oj1 + ring, m1);
    const int w = a1 - a0, n = w * (b1 - b0);
    const bool first = pre && s == 1;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const int jj = t / w;
      const int i = a0 + (t - jj * w), j = b0 + jj;
      if (((i + j) & 1) != col) continue;
      const int c = (i - B.i0) + B.rx * (j - B.j0);
      T v = S.b[c];
      if (!first) {
        if (i > 0) v += S.c0[c] * S.x[c - 1];
        if (i < m0 - 1) v += S.c0[c + 1] * S.x[c + 1];
        if (j > 0) v += S.c1[c] * S.x[c - B.rx];
        if (j < m1 - 1) v += S.c1[c + B.rx] * S.x[c + B.rx];
      }
      S.x[c] = v * S.idg[c];
    }
    __syncthreads();
  }
}

// operator of a tile region into shared memory (with D: for the residual)
template <typename T>
__device__ __forceinline__ void tile_load_op(const TileSmem<T>& S, const TileBox& B, const LevV<T>& F, int c,
                                             long long g, bool withD = false) {
  S.idg[c] = F.idg[g];
  S.c0[c] = F.c[0][g];
  S.c1[c] = F.c[1][g];
  if (withD) S.D[c] = F.D[g];
}

// residual b - A x of the owned cells of a pre-smoothed tile, restricted (summed over
// each 2 x 2 aggregate) into C.b: mg_resid's arithmetic and grid_restrict's order on
// the values the tile holds
template <typename T>
__device__ void tile_restrict(const TileSmem<T>& S, const TileBox& B, int m0, int m1, const LevV<T>& C) {
  const int cw = (B.oi1 - B.oi0) / 2, n = cw * ((B.oj1 - B.oj0) / 2);
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int JJ = t / cw;
    const int I = B.oi0 / 2 + (t - JJ * cw), J = B.oj0 / 2 + JJ;
    T s = 0;
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        const int i = 2 * I + di, j = 2 * J + dj;
        const int c = (i - B.i0) + B.rx * (j - B.j0);
        const T xp = S.x[c];
        T y = S.D[c] * xp;
        if (i > 0) y += S.c0[c] * (xp - S.x[c - 1]);
        if (i < m0 - 1) y += S.c0[c + 1] * (xp - S.x[c + 1]);
        if (j > 0) y += S.c1[c] * (xp - S.x[c - B.rx]);
        if (j < m1 - 1) y += S.c1[c + B.rx] * (xp - S.x[c + B.rx]);
        s += S.b[c] - y;
      }
    ((T*)C.b)[(long long)I + (long long)C.m[0] * J] = s;
  }
}

template <typename T>
__device__ __forceinline__ void tile_store_x(const TileSmem<T>& S, const TileBox& B, int m0, T* dst) {
  const int w = B.oi1 - B.oi0, n = w * (B.oj1 - B.oj0);
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int jj = t / w;
    const int i = B.oi0 + (t - jj * w), j = B.oj0 + jj;
    dst[(long long)i + (long long)m0 * j] = S.x[(i - B.i0) + B.rx * (j - B.j0)];
  }
}

// pre-smoothing of a 2D level l >= 1 (b from the restriction), tile by tile, and the
// restriction of its residual into C.b
template <typename T>
__device__ void tiled_pre(const TileSmem<T>& S, const LevV<T>& F, const LevV<T>& C, int TX, int TY) {
  const int m0 = F.m[0], m1 = F.m[1];
  for (int t = blockIdx.x; t < tile_count(m0, m1, TX, TY); t += gridDim.x) {
    const TileBox B = tile_box(m0, m1, t, TX, TY);
    const int n = B.rx * B.ry;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const int lj = c / B.rx;
      const long long g = (long long)(B.i0 + c - lj * B.rx) + (long long)m0 * (B.j0 + lj);
      S.b[c] = F.b[g];
      tile_load_op<T>(S, B, F, c, g, true);
    }
    __syncthreads();
    tile_sweeps<T>(S, B, m0, m1, true);
    tile_store_x<T>(S, B, m0, F.x);
    tile_restrict<T>(S, B, m0, m1, C);
    __syncthreads();
  }
}

// prolongation and post-smoothing of a 2D level, tile by tile: reads the pre-smoothed
// F.x and the coarse level's final iterate cx, writes F.xp (tiles of other blocks
// still read F.x in their halos during the phase)
template <typename T>
__device__ void tiled_post(const TileSmem<T>& S, const LevV<T>& F, const LevV<T>& C, const T* cx, int TX, int TY) {
  const int m0 = F.m[0], m1 = F.m[1];
  for (int t = blockIdx.x; t < tile_count(m0, m1, TX, TY); t += gridDim.x) {
    const TileBox B = tile_box(m0, m1, t, TX, TY);
    const int n = B.rx * B.ry;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const int lj = c / B.rx;
      const int i = B.i0 + c - lj * B.rx, j = B.j0 + lj;
      const long long g = (long long)i + (long long)m0 * j;
      S.x[c] = prolonged<T>(F, C, cx, g, i, j, 0);
      S.b[c] = F.b[g];
      tile_load_op<T>(S, B, F, c, g);
    }
    __syncthreads();
    tile_sweeps<T>(S, B, m0, m1, false);
    tile_store_x<T>(S, B, m0, F.xp);
    __syncthreads();
  }
}

template <typename T>
struct MgArgs {
  BoxV A;                      // FP64 pressure operator
  const double* b;             // right-hand side
  double tol2;                 // rtol^2
  int maxit;
  int cast0;                   // level 0 holds FP32 copies of the operator
  RecordSpec rec;
  double* x;                   // initial guess in, solution out
  double *r[2], *q[2];         // residual and q = A p, double buffered (tiles read neighbours')
  double *p, *w;               // direction, w = A z
  TailLevels<T> TL;            // hierarchy views and the tail's shared-memory layout
  const T* z0;                 // level-0 iterate at the end of a V-cycle (z = M r)
  int tx, ty;                  // tile shape of the temporal blocking
  int nlev, lt, ncoarse;       // levels, first tail level, coarsest-level sweeps
  int dn, dw, dp;              // dense coarsest level: cells (0: swept), smem offsets of W and sums
  double* part;
  double* stat;
  int* done;
  unsigned* bar;
  int* err;
  long long spin;              // polls of a grid-barrier wait before it gives up
};

// Phase A on a 2D level 0: the CG update (x, p of the tile's cells; r and q of the
// tile region into the other buffers, halo cells recomputed from the neighbours'
// current values), b = r, the whole pre-smoothing of the tile and the restriction of
// its residual into level 1.  Returns the block's share of |r_new|^2 over its owned
// cells.
template <typename T>
__device__ double tiled_phase_a(const TileSmem<T>& S, const MgArgs<T>& a, int cur, int its, double alpha,
                                double beta) {
  const LevV<T>& L0 = a.TL.L[0];
  const int m0 = L0.m[0], m1 = L0.m[1];
  const double *r = a.r[cur], *q = a.q[cur];
  double *rn = a.r[cur ^ 1], *qn = a.q[cur ^ 1];
  double rr = 0.0;
  const int TX = a.tx, TY = a.ty;
  for (int t = blockIdx.x; t < tile_count(m0, m1, TX, TY); t += gridDim.x) {
    const TileBox B = tile_box(m0, m1, t, TX, TY);
    const int n = B.rx * B.ry;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const int lj = c / B.rx;
      const int i = B.i0 + c - lj * B.rx, j = B.j0 + lj;
      const long long g = (long long)i + (long long)m0 * j;
      double rP = r[g];
      const bool own = i >= B.oi0 && i < B.oi1 && j >= B.oj0 && j < B.oj1;
      if (its > 0) {
        const double qP = its > 1 ? a.w[g] + beta * q[g] : a.w[g];   // q_old = 0 at the start
        rP -= alpha * qP;
        if (own) {
          const double zP = (double)a.z0[g];
          const double pP = its > 1 ? zP + beta * a.p[g] : zP;
          a.p[g] = pP;
          a.x[g] += alpha * pP;
          qn[g] = qP;
          rn[g] = rP;
          rr += rP * rP;
        }
      }
      const T bP = (T)rP;
      S.b[c] = bP;
      if (own) ((T*)L0.b)[g] = bP;
      tile_load_op<T>(S, B, L0, c, g, true);
    }
    __syncthreads();
    tile_sweeps<T>(S, B, m0, m1, true);
    tile_store_x<T>(S, B, m0, L0.x);
    tile_restrict<T>(S, B, m0, m1, a.TL.L[1]);
    __syncthreads();
  }
  return rr;
}

template <typename T>
__global__ void __launch_bounds__(PTPB, 1) k_mgpcg_persist(MgArgs<T> a) {
  extern __shared__ __align__(16) unsigned char pmg_smem[];
  T* sm = reinterpret_cast<T*>(pmg_smem);
  TileSmem<T> S;
  {
    T* tb = sm + (a.TL.total + 3) / 4 * 4;
    const int treg = tile_region(a.tx, a.ty);
    S.x = tb;
    S.b = tb + treg;
    S.idg = tb + 2 * treg;
    S.c0 = tb + 3 * treg;
    S.c1 = tb + 4 * treg;
    S.D = tb + 5 * treg;
  }
  __shared__ double bc[2];
  const int gs = gridDim.x * blockDim.x;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const LevV<T>& L0 = a.TL.L[0];
  const long long N = a.A.N;
  const int maxit = a.maxit, lt = a.lt;
  int phase = 0, its = 0, result = 2, cur = 0;
  auto sync = [&](double (&v)[3], int nv) { return grid_sum3<double>(v, nv, phase++, a.part, a.bar, a.err, a.spin); };
  // phase H0: r0 = b - A x0 in FP64, |b|^2 and |r0|^2; the level-0 operator in the
  // hierarchy precision and its 1 / diag
  double h[3] = {0.0, 0.0, 0.0};
  for (long long id = gid; id < N; id += gs) {
    int i, j, k;
    bdecomp(a.A.m, id, i, j, k);
    double ax, dt;
    box_row<double, double, false>(a.A.m, a.A.D, a.A.c, a.x, id, i, j, k, ax, dt);
    const double bP = a.b[id], r0 = bP - ax;
    a.r[0][id] = r0;
    h[0] += bP * bP;
    h[1] += r0 * r0;
    if (a.cast0) {
      ((T*)L0.D)[id] = (T)a.A.D[id];
      for (int q = 0; q < 3; ++q)
        if (a.A.c[q]) ((T*)L0.c[q])[id] = (T)a.A.c[q][id];
    }
    // 1 / diag from the values as the level holds them (FP32 copies or the FP64 box)
    LevV<T> V = L0;
    double dd = (double)(T)a.A.D[id];
    {
      long long st[3] = {1, (long long)V.m[0], (long long)V.m[0] * V.m[1]};
      int qq[3] = {i, j, k};
      for (int q = 0; q < 3; ++q) {
        if (!a.A.c[q] || V.m[q] < 2) continue;
        if (qq[q] > 0) dd += (double)(T)a.A.c[q][id];
        if (qq[q] < V.m[q] - 1) dd += (double)(T)a.A.c[q][id + st[q]];
      }
    }
    ((T*)L0.idg)[id] = (T)(1.0 / dd);
  }
  bool ok = sync(h, 2);
  const double bb = h[0], thr = a.tol2 * bb;
  double alpha = 0.0, beta = 0.0, gamma = 1.0, rr_last = h[1];
  if (!ok) result = 3;
  else if (bb == 0.0 || h[1] <= thr) result = 1;     // converged at the initial guess
  // the coarse levels: level l coarsened from l - 1 together with 1 / diag of l - 1
  for (int l = 1; ok && result != 1 && l <= a.nlev; ++l) {
    if (l < a.nlev) {
      const LevV<T>& F = a.TL.L[l - 1];
      const LevV<T>& C = a.TL.L[l];
      for (long long id = gid; id < C.N; id += gs)
        mg_coarsen_cell<T>(F, C, id, (T*)C.D, (T*)C.c[0], (T*)C.c[1], (T*)C.c[2]);
    }
    if (l >= 2) {
      const LevV<T>& P = a.TL.L[l - 1];
      for (long long id = gid; id < P.N; id += gs) ((T*)P.idg)[id] = mg_idg_cell<T>(P, id);
    }
    if (l < a.nlev || l >= 2) ok = sync(h, 0);
    if (!ok) result = 3;
  }
  // the dense coarsest level, factored once per solve by block 0 (tile arrays as scratch)
  DenseCoarse<T> dc{nullptr, nullptr, 0};
  if (blockIdx.x == 0 && a.dn > 0 && ok && result != 1) {
    if (dense_factor<T>(a.TL.L[a.nlev - 1], a.dn, sm + a.dw, S.x)) dc = DenseCoarse<T>{sm + a.dw, sm + a.dp, a.dn};
  }
  for (; ok && result != 1;) {
    double v[3] = {0.0, 0.0, 0.0};
    const bool tiled0 = lt > 0 && L0.m[2] == 1;
    // phase A: CG update, level-0 right-hand side and the start of the pre-smoothing
    if (tiled0) {
      v[0] = tiled_phase_a<T>(S, a, cur, its, alpha, beta);
    } else {
      const double *r = a.r[cur], *q = a.q[cur];
      double *rn = a.r[cur ^ 1], *qn = a.q[cur ^ 1];
      for (long long id = gid; id < N; id += gs) {
        double rP = r[id];
        if (its > 0) {
          const double zP = (double)a.z0[id];
          const double pP = its > 1 ? zP + beta * a.p[id] : zP;   // p_old = q_old = 0 at the start
          const double qP = its > 1 ? a.w[id] + beta * q[id] : a.w[id];
          a.p[id] = pP;
          qn[id] = qP;
          a.x[id] += alpha * pP;
          rP -= alpha * qP;
          rn[id] = rP;
          v[0] += rP * rP;
        }
        const T bP = (T)rP;
        ((T*)L0.b)[id] = bP;
        if (lt > 0) {
          int i, j, k;
          bdecomp(L0.m, id, i, j, k);
          if (((i + j + k) & 1) == 0) L0.x[id] = bP * L0.idg[id];
        }
      }
    }
    if (!sync(v, its > 0 ? 1 : 0)) { result = 3; break; }
    if (its > 0) {
      cur ^= 1;
      rr_last = v[0];
      if (v[0] <= thr) { result = 1; break; }
    }
    if (its >= maxit) break;
    // V-cycle down: pre-smoothing and restriction on the grid levels
    bool ok = true;
    for (int l = 0; l < lt && ok; ++l) {
      const LevV<T>& F = a.TL.L[l];
      const LevV<T>& C = a.TL.L[l + 1];
      if (F.m[2] > 1) {   // 3D: level-wide half sweeps (the red half sweep of sweep 0
                          // came before), then the restriction with C's first red half sweep
        for (int s = 0; s < MG_NU && ok; ++s) {
          if (s > 0) {
            grid_half_sweep<T>(F, 0, 0, gid, gs);
            ok = sync(v, 0);
          }
          grid_half_sweep<T>(F, 1, 0, gid, gs);
          ok = ok && sync(v, 0);
        }
        if (!ok) break;
        grid_restrict<T>(F, C, l + 1 < lt, gid, gs);
        ok = sync(v, 0);
        continue;
      }
      // 2D: F's tiled phase restricted into C.b; C's own tiled phase restricts further
      if (l + 1 < lt) {
        tiled_pre<T>(S, C, a.TL.L[l + 2], a.tx, a.ty);
        ok = sync(v, 0);
      }
    }
    if (!ok) { result = 3; break; }
    // the tail levels in block 0, out of shared memory
    if (blockIdx.x == 0) tail_vcycle<T>(a.TL, sm, lt, a.nlev, MG_NU, a.ncoarse, dc);
    if (!sync(v, 0)) { result = 3; break; }
    // V-cycle up: prolongation and post-smoothing on the grid levels
    for (int l = lt - 1; l >= 0 && ok; --l) {
      const LevV<T>& F = a.TL.L[l];
      if (F.m[2] == 1) {
        const LevV<T>& C = a.TL.L[l + 1];
        tiled_post<T>(S, F, C, l + 1 < lt ? C.xp : C.x, a.tx, a.ty);
        ok = sync(v, 0);
        continue;
      }
      grid_prolong_black<T>(F, a.TL.L[l + 1], gid, gs);
      ok = sync(v, 0);
      grid_half_sweep<T>(F, 0, 0, gid, gs);
      ok = ok && sync(v, 0);
      for (int s = 1; s < MG_NU && ok; ++s) {
        grid_half_sweep<T>(F, 1, 0, gid, gs);
        ok = sync(v, 0);
        grid_half_sweep<T>(F, 0, 0, gid, gs);
        ok = ok && sync(v, 0);
      }
    }
    if (!ok) { result = 3; break; }
    // phase W: z = M r (level-0 x), w = A z, gamma = r.z, delta = w.z
    v[0] = v[1] = v[2] = 0.0;
    {
      const double* r = a.r[cur];
      for (long long id = gid; id < N; id += gs) {
        int i, j, k;
        bdecomp(a.A.m, id, i, j, k);
        double wP, dtot;
        box_row<double, T, false>(a.A.m, a.A.D, a.A.c, a.z0, id, i, j, k, wP, dtot);
        const double zP = (double)a.z0[id];
        a.w[id] = wP;
        v[0] += r[id] * zP;
        v[1] += wP * zP;
      }
    }
    if (!sync(v, 2)) { result = 3; break; }
    if (threadIdx.x == 0) {
      if (its == 0) {
        bc[0] = v[0] / v[1];
        bc[1] = 0.0;
      } else {
        const double bn = v[0] / gamma;
        bc[0] = v[0] / (v[1] - bn * v[0] / alpha);
        bc[1] = bn;
      }
    }
    __syncthreads();
    alpha = bc[0];
    beta = bc[1];
    gamma = v[0];
    __syncthreads();
    ++its;
  }
  persist_finish(a.stat, a.done, a.rec, its, rr_last, bb, result, a.bar, a.err, a.rec.scal);
}

template <typename TO, typename TI>
__global__ void k_cast(long long n, TO* y, const TI* x) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id < n) y[id] = (TO)x[id];
}
template <typename TO, typename TI>
__global__ void k_cast_done(long long n, TO* y, const TI* x, const int* done) {
  if (*done) return;
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id < n) y[id] = (TO)x[id];
}

// ---------------------------------------------------------------- host side
long long g_launches = 0;

int Prof::begin(int k, cudaStream_t st, double b, double f64) {
  if (2 * (used + 1) > pool.size()) {
    for (int q = 0; q < 256; ++q) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      pool.push_back(e);
    }
  }
  int idx = (int)used++;
  if ((int)kind.size() < (int)used) kind.resize(used);
  kind[idx] = k;
  bytes[k] += b;
  flops[k] += f64;
  n[k] += 1;
  cudaEventRecord(pool[2 * idx], st);
  return idx;
}

void Prof::end(int idx, cudaStream_t st) { cudaEventRecord(pool[2 * idx + 1], st); }

void Prof::reset() {
  used = 0;
  for (int k = 0; k < KC_COUNT; ++k) { bytes[k] = 0.0; flops[k] = 0.0; n[k] = 0; }
}

int Prof::read(int k, double* ms, long long* launches, double* bytes_total, double* flops_total) {
  double tot = 0.0;
  for (size_t i = 0; i < used; ++i) {
    if (kind[i] != k) continue;
    float t = 0.f;
    if (cudaEventSynchronize(pool[2 * i + 1]) != cudaSuccess) return DROPLET_ERR_CUDA;
    if (cudaEventElapsedTime(&t, pool[2 * i], pool[2 * i + 1]) != cudaSuccess) return DROPLET_ERR_CUDA;
    tot += t;
  }
  *ms = tot;
  *launches = n[k];
  *bytes_total = bytes[k];
  if (flops_total) *flops_total = flops[k];
  return 0;
}

void Prof::destroy() {
  for (auto e : pool) cudaEventDestroy(e);
  pool.clear();
  kind.clear();
  used = 0;
}
#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { fprintf(stderr, "droplet: %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); return DROPLET_ERR_CUDA; } } while (0)

int Solver::setup(long long maxN, cudaStream_t s) {
  stream = s;
  cap = maxN;
  size_t b = sizeof(double) * (size_t)maxN;
  CK(cudaMalloc(&r, b));
  CK(cudaMalloc(&z, b));
  CK(cudaMalloc(&p, b));
  CK(cudaMalloc(&Ap, b));
  CK(cudaMalloc(&idg, b));
  CK(cudaMalloc(&adg, b));
  CK(cudaMalloc(&part, sizeof(double) * RED_BLOCKS * 8));
  CK(cudaMalloc(&sc, sizeof(double) * S_COUNT));
  CK(cudaMalloc(&done, sizeof(int)));
  CK(cudaMalloc(&cnt, sizeof(unsigned)));
  CK(cudaMemset(cnt, 0, sizeof(unsigned)));
  CK(cudaMallocHost(&hsc, sizeof(double) * (S_COUNT + 2)));
  CK(cudaMalloc(&bar, 2 * sizeof(unsigned)));
  CK(cudaMemset(bar, 0, 2 * sizeof(unsigned)));
  CK(cudaMalloc(&err, sizeof(int)));
  CK(cudaMemset(err, 0, sizeof(int)));
  if (f32_helm) {
    size_t bf = sizeof(float) * (size_t)maxN;
    float** fa[] = {&fD, &fc[0], &fc[1], &fc[2], &fidg, &fr, &fz, &fp, &fAp, &fdx};
    for (auto q : fa) CK(cudaMalloc((void**)q, bf));
  }
  if (persistent) CK(cudaMalloc(&mg_q2, sizeof(double) * (size_t)maxN));
  if (persist_pcg)
    for (int k = 0; k < nsys_extra; ++k)
      for (int q = 0; q < PERSIST_VECTORS; ++q)
        CK(cudaMalloc(&pwx[k][q], (f32_helm ? sizeof(float) : sizeof(double)) * (size_t)maxN));
  if (persist_pcg)
    for (int q = 0; q < PERSIST_VECTORS; ++q) CK(cudaMalloc(&pw[q], (f32_helm ? sizeof(float) : sizeof(double)) * (size_t)maxN));
  return 0;
}

void Solver::release() {
  cudaFree(r); cudaFree(z); cudaFree(p); cudaFree(Ap); cudaFree(idg); cudaFree(adg);
  adg = nullptr;
  cudaFree(part); cudaFree(sc); cudaFree(done); cudaFree(cnt); cudaFreeHost(hsc);
  {
    float** fa[] = {&fD, &fc[0], &fc[1], &fc[2], &fidg, &fr, &fz, &fp, &fAp, &fdx};
    for (auto q : fa) { cudaFree(*q); *q = nullptr; }
    for (int q = 0; q < PERSIST_VECTORS; ++q) { cudaFree(pw[q]); pw[q] = nullptr; }
    for (int k = 0; k < 2; ++k)
      for (int q = 0; q < PERSIST_VECTORS; ++q) { cudaFree(pwx[k][q]); pwx[k][q] = nullptr; }
    cudaFree(bar); cudaFree(err); cudaFree(mg_q2);
    mg_q2 = nullptr;
    bar = nullptr; err = nullptr;
  }
  cnt = nullptr;
  cudaFree(mgbuf);
  r = z = p = Ap = idg = part = sc = nullptr;
  done = nullptr; hsc = nullptr; mgbuf = nullptr;
}

static BoxV view(const BoxSys& s) {
  BoxV v;
  for (int a = 0; a < 3; ++a) { v.m[a] = s.m[a]; v.c[a] = s.c[a]; }
  v.N = s.N;
  v.D = s.D;
  return v;
}

// read the device status; returns 1 when the solve stopped (converged or capped)
static int poll(double* hsc, const double* sc, const int* done, cudaStream_t st, int maxit, int* conv) {
  cudaMemcpyAsync(hsc, sc, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(hsc + S_COUNT, done, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  int d = *(int*)(hsc + S_COUNT);
  *conv = d == 1;
  return d != 0 || (int)hsc[S_ITS] >= maxit;
}

// status of a persistent solve after poll(): a wait that ran out before not converging
static int persist_status(const double* hsc, int conv) {
  if (hsc[S_TMO] != 0.0) return DROPLET_ERR_TIMEOUT;
  return conv ? 0 : DROPLET_ERR_NOT_CONVERGED;
}

static void fill_stats(const double* hsc, int conv, SolveStats* out) {
  if (!out) return;
  out->its = (int)hsc[S_ITS];
  out->relres = hsc[S_BB] > 0 ? sqrt(hsc[S_RR] / hsc[S_BB]) : 0.0;
  out->converged = conv;
}

void Solver::record(double* scal, int slot_its, int slot_res, int accumulate) {
  rec_scal = nullptr;   // a launched solve does not consume the slots set for it
  if (recorded) {       // the persistent solve wrote its statistics itself
    recorded = false;
    return;
  }
  ++g_launches, k_record<<<1, 1, 0, stream>>>(sc, done, scal, slot_its, slot_res, accumulate);
}

RecordSpec Solver::take_record() {
  RecordSpec r{rec_scal, rec_its, rec_res, rec_acc};
  recorded = rec_scal != nullptr;
  rec_scal = nullptr;
  return r;
}

// Inside a stream capture: a conditional WHILE node whose body is one solver
// iteration (captured from `body` on stream2) followed by the condition update.
// The loop ends when the done flag is set: converged, or the iteration cap.
template <typename F>
int Solver::device_loop(F body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(stream, &cs, nullptr, &g, &deps, &ed, &nd));
  if (cs != cudaStreamCaptureStatusActive) return DROPLET_ERR_CUDA;
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
  ++g_launches, k_set_cond<<<1, 1, 0, stream>>>(h, done);
  CK(cudaStreamGetCaptureInfo(stream, &cs, nullptr, &g, &deps, &ed, &nd));
  // the parameter struct holds a union without a default constructor: zeroed raw storage
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams* np = reinterpret_cast<cudaGraphNodeParams*>(raw);
  np->type = cudaGraphNodeTypeConditional;
  np->conditional.handle = h;
  np->conditional.type = cudaGraphCondTypeWhile;
  np->conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, deps, ed, nd, np));
  cudaGraph_t bodyg = np->conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(stream2, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  cudaStream_t saved = stream;
  stream = stream2;
  body();
  ++g_launches, k_set_cond<<<1, 1, 0, stream>>>(h, done);
  stream = saved;
  CK(cudaStreamEndCapture(stream2, &bodyg));
  CK(cudaStreamUpdateCaptureDependencies(stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return 0;
}

template <typename T>
int Solver::pcg_persist(const BoxSys* sys, int K, double rtol, int maxit, const RecordSpec* recs, SolveStats* out) {
  constexpr bool f32 = sizeof(T) == 4;
  PersistMulti<T> M;
  memset(&M, 0, sizeof(M));
  M.K = K;
  long long nmax = 0;
  double setup_b = 0.0, iter_b[PMAXSYS] = {0.0, 0.0, 0.0};
  for (int k = 0; k < K; ++k) {
    const BoxSys& s = sys[k];
    PersistArgs<T>& a = M.s[k];
    void* const* v = k == 0 ? pw : pwx[k - 1];
    a.A = view(s);
    a.b = s.b;
    a.x = s.x;
    a.tol2 = rtol * rtol;
    a.maxit = maxit;
    a.rec = recs[k];
    for (int q = 0; q < 3; ++q) a.ch[q] = (T*)v[q];
    a.dg = (T*)v[3];
    a.sc = (T*)v[4];
    for (int q = 0; q < 2; ++q) {
      a.r[q] = (T*)v[5 + q];
      a.s[q] = (T*)v[7 + q];
      a.w[q] = (T*)v[9 + q];
    }
    a.p = (T*)v[11];
    a.dx = (T*)v[12];
    nmax = std::max(nmax, s.N);
    // algorithmic bytes: setup (FP64 operator read twice and defect in; diag, S, r^, s,
    // p, x^, c^, w out), the final x += S x^ / nu, and per iteration r^, s, w, p, x^,
    // diag and c^ in, r^, s, w, p, x^ out
    const double na = s.c[2] ? 3.0 : 2.0, wb = (double)sizeof(T);
    setup_b += ((2.0 + 2.0 * na) * 8.0 + (7.0 + na) * wb + 2.0 * wb + 16.0) * s.N;
    iter_b[k] = (11.0 + na) * wb * s.N;
  }
  M.stat = sc;
  M.done = done;
  M.bar = bar;
  M.err = err;
  M.spin = spin_limit;
  M.split = nmax >= PERSIST_SPLIT_CELLS;
  int grid = (int)((nmax + PTPB - 1) / PTPB);
  int cap = persist_blocks(f32);
  const int bud = pcg_budget > 0 ? pcg_budget : sm_budget;
  if (bud > 0) cap = std::min(cap, bud * std::max(1, cap / nsm_));
  if (grid > cap) grid = cap;
  // partials in `part` (8 RED_BLOCKS doubles): the FP64 initial norms (2 x 2 PMAXSYS per
  // block) first, then the sums of precision T (2 x 3 PMAXSYS per block)
  const int per_blk = 4 * PMAXSYS + (f32 ? 3 * PMAXSYS : 6 * PMAXSYS);   // doubles per block
  if (grid > 8 * RED_BLOCKS / per_blk) grid = 8 * RED_BLOCKS / per_blk;
  if (grid < 1) grid = 1;
  M.part64 = part;
  M.part = (T*)(part + 4 * PMAXSYS * grid);
  cudaLaunchConfig_t lc;
  memset(&lc, 0, sizeof(lc));
  lc.gridDim = dim3(grid);
  lc.blockDim = dim3(PTPB);
  lc.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  ++g_launches;
  {
    ProfScope ps(prof, KC_PCG_PERSIST, stream, setup_b);
    CK(cudaLaunchKernelEx(&lc, k_pcg_persist<T>, M));
  }
  if (capturing) return 0;
  int conv = 0;
  poll(hsc, sc, done, stream, maxit, &conv);
  // (each system's iterations times its bytes per iteration)
  if (prof && prof->on)
    for (int k = 0; k < K; ++k) prof->bytes[KC_PCG_PERSIST] += hsc[S_ITSK + k] * iter_b[k];
  fill_stats(hsc, conv, out);
  return persist_status(hsc, conv);
}

int Solver::pcg_jacobi_multi(const BoxSys* s, int K, double rtol, int maxit, const RecordSpec* recs,
                             SolveStats* out) {
  if (!persist_pcg || K < 1 || K > 1 + nsys_extra) return DROPLET_ERR_ARG;
  recorded = false;
  rec_scal = nullptr;
  return f32_helm ? pcg_persist<float>(s, K, rtol, maxit, recs, out) : pcg_persist<double>(s, K, rtol, maxit, recs, out);
}

int Solver::persist_blocks(bool f32) {
  int& cache = f32 ? pb_f32 : pb_f64;
  if (cache > 0) return cache;
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  nsm_ = nsm;
  if (f32) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_persist<float>, PTPB, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_persist<double>, PTPB, 0);
  cache = per * nsm;
  return cache;
}

int Solver::cg_grid(long long N) {
  if (nsm_ <= 1) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm > 0) nsm_ = nsm;
  }
  return std::min(red_grid_cap(N, rb), CG_BLOCKS_PER_SM * nsm_);
}

int Solver::pcg_jacobi(const BoxSys& s, double rtol, int maxit, SolveStats* out) {
  if (persist_pcg) {
    const RecordSpec rec = take_record();
    return f32_helm ? pcg_persist<float>(&s, 1, rtol, maxit, &rec, out) : pcg_persist<double>(&s, 1, rtol, maxit, &rec, out);
  }
  if (f32_helm) return pcg_jacobi_f32(s, rtol, maxit, out);
  BoxV A = view(s);
  int nb = cg_grid(s.N);
  ++g_launches, k_pcg_init<<<nb, TPB, 0, stream>>>(A, s.b, s.x, r, z, p, idg, 1, part, adg);
  ++g_launches, k_fin_init<<<1, TPB, 0, stream>>>(part, nb, sc, done, rtol * rtol, maxit, nullptr, nullptr);
  auto iteration = [&]() {
    {
      ProfScope ps(prof, KC_SPMV, stream, (3.0 + (s.c[2] ? 3 : 2)) * s.N * 8.0, (2.0 * (s.c[2] ? 3 : 2) + 2.0) * s.N);
      ++g_launches, k_spmv_dot<<<nb, TPB, 0, stream>>>(A, p, Ap, part, done, sc, cnt, adg);
    }
    {
      ProfScope ps(prof, KC_UPDATE, stream, 8.0 * s.N * 8.0, 5.0 * s.N);
      ++g_launches, k_update<<<nb, TPB, 0, stream>>>(s.N, s.x, r, p, Ap, idg, z, 1, sc, part, done, cnt);
    }
    ++g_launches, k_p_update<<<red_grid_cap(s.N, rb), TPB, 0, stream>>>(s.N, p, z, sc, done);
  };
  if (capturing) return device_loop(iteration);
  // the host polls after every chunk of iterations; while the kernel classes are timed it
  // polls after each one, so that no timed launch is one that returned at once
  const int chunk = (prof && prof->on) ? 1 : 8;
  int conv = 0;
  for (int it = 0; it < maxit; it += chunk) {
    for (int q = 0; q < chunk; ++q) iteration();
    CK(cudaGetLastError());
    if (poll(hsc, sc, done, stream, maxit, &conv)) break;
  }
  if (!conv) poll(hsc, sc, done, stream, maxit, &conv);
  fill_stats(hsc, conv, out);
  return conv ? 0 : DROPLET_ERR_NOT_CONVERGED;
}

int Solver::pcg_jacobi_f32(const BoxSys& s, double rtol, int maxit, SolveStats* out) {
  BoxV A = view(s);
  BoxVf Af;
  for (int a = 0; a < 3; ++a) { Af.m[a] = s.m[a]; Af.c[a] = s.c[a] ? fc[a] : nullptr; }
  Af.N = s.N;
  Af.D = fD;
  int nb = cg_grid(s.N);
  // FP64 defect of the initial guess, ||b||, ||r0||
  ++g_launches, k_pcg_init<<<nb, TPB, 0, stream>>>(A, s.b, s.x, r, z, p, idg, 0, part);
  ++g_launches, k_fin_init<<<1, TPB, 0, stream>>>(part, nb, sc, done, rtol * rtol, maxit, nullptr, nullptr);
  ++g_launches, k_mx_setup<<<nb, TPB, 0, stream>>>(A, r, fD, fc[0], fc[1], s.c[2] ? fc[2] : fc[0], fidg, fr, fz, fp, fdx,
                                                  part, done, sc, cnt);
  auto iteration = [&]() {
    {
      ProfScope ps(prof, KC_SPMV, stream, (3.0 + (s.c[2] ? 3 : 2)) * s.N * 4.0);
      ++g_launches, k_spmv_f<<<nb, TPB, 0, stream>>>(Af, fp, fAp, part, done, sc, cnt);
    }
    {
      ProfScope ps(prof, KC_UPDATE, stream, 8.0 * s.N * 4.0);
      ++g_launches, k_update_f<<<nb, TPB, 0, stream>>>(s.N, fdx, fr, fp, fAp, fidg, fz, sc, part, done, cnt);
    }
    ++g_launches, k_p_update_f<<<nb, TPB, 0, stream>>>(s.N, fp, fz, sc, done);
  };
  int rc = 0;
  if (capturing) {
    rc = device_loop(iteration);
  } else {
    int conv = 0;
    const int chunk = (prof && prof->on) ? 1 : 8;
    for (int it = 0; it < maxit; it += chunk) {
      for (int q = 0; q < chunk; ++q) iteration();
      CK(cudaGetLastError());
      if (poll(hsc, sc, done, stream, maxit, &conv)) break;
    }
    if (!conv) poll(hsc, sc, done, stream, maxit, &conv);
    fill_stats(hsc, conv, out);
    rc = conv ? 0 : DROPLET_ERR_NOT_CONVERGED;
  }
  ++g_launches, k_mx_finish<<<lin_grid(s.N), TPB, 0, stream>>>(s.N, s.x, fdx, sc);
  return rc;
}

// ---------------------------------------------------------------- multigrid setup / cycle
template <typename T>
static LevV<T> lv(const MGLevel& L) {
  LevV<T> v;
  for (int a = 0; a < 3; ++a) { v.m[a] = L.m[a]; v.c[a] = (const T*)L.c[a]; }
  v.N = L.N;
  v.D = (const T*)L.D;
  v.x = (T*)L.x;
  v.b = (const T*)L.b;
  v.idg = (const T*)L.idg;
  v.xp = (T*)L.xp;
  v.split = L.split;
  v.bs = (T*)L.xp;   // (xp serves only the persistent V-cycle; the launched one keeps b there)
  return v;
}

int Solver::prepare_mg(const int mm[3], int fp32) {
  size_t es = fp32 ? sizeof(float) : sizeof(double);
  if (mg_fp32 == fp32 && mg_m[0] == mm[0] && mg_m[1] == mm[1] && mg_m[2] == mm[2]) return 0;
  // level dims: halve while every active dim is even and > 2
  int m[3] = {mm[0], mm[1], mm[2]};
  bool d3 = mm[2] > 1;
  nlev = 0;
  size_t total = 0;
  for (;;) {
    MGLevel& L = lev[nlev];
    for (int a = 0; a < 3; ++a) L.m[a] = m[a];
    L.N = (long long)m[0] * m[1] * m[2];
    total += (size_t)L.N * es * 8;
    nlev++;
    bool can = (m[0] % 2 == 0 && m[1] % 2 == 0 && m[0] > 2 && m[1] > 2) && (!d3 || (m[2] % 2 == 0 && m[2] > 2));
    if (!can || nlev >= 24) break;
    m[0] /= 2; m[1] /= 2;
    if (d3) m[2] /= 2;
  }
  cudaFree(mgbuf);
  mgbuf = nullptr;
  CK(cudaMalloc(&mgbuf, total + 256 * 8 * nlev));
  char* ptr = (char*)mgbuf;
  auto take = [&](long long n) { void* q = ptr; ptr += ((size_t)n * es + 255) / 256 * 256; return q; };
  for (int l = 0; l < nlev; ++l) {
    MGLevel& L = lev[l];
    L.D = take(L.N);
    L.c[0] = take(L.N);
    L.c[1] = take(L.N);
    L.c[2] = d3 ? take(L.N) : nullptr;
    L.x = take(L.N);
    L.b = take(L.N);
    L.idg = take(L.N);
    L.xp = take(L.N);
  }
  // shared memory of the one-block tail of the V-cycle
  int lt = nlev - 1;
  while (lt > 0 && lev[lt - 1].N <= TAIL_MAX_CELLS) --lt;
  // (the limit is raised to the device's opt-in maximum, not to this hierarchy's need,
  // so that contexts with different hierarchies do not lower it for one another)
  const size_t smem = (size_t)tail_layout(lev, lt, nlev, es, nullptr, nullptr) * es;
  int dev = 0, optin = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem > (size_t)optin) return DROPLET_ERR_SIZE;
  if (fp32) CK(cudaFuncSetAttribute(k_mg_tail<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  else CK(cudaFuncSetAttribute(k_mg_tail<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
  if (persistent) {
    // the persistent MG-PCG: its own (smaller) tail; co-resident blocks at that size
    int ltp = nlev - 1;
    while (ltp > 0 && lev[ltp - 1].N <= PMG_TAIL_MAX_CELLS) --ltp;
    const int lcp = dense_level(lev, ltp, nlev, fp32);
    const int nlp = lcp >= 0 ? lcp + 1 : nlev;
    const size_t psm = pmg_layout((int)tail_layout(lev, ltp, nlp, es, nullptr, nullptr), es, 32, 32,
                                  lcp >= 0 ? (int)lev[lcp].N : 0).bytes;
    int nsm = 0, per = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // (dynamic limit: the opt-in maximum less the kernel's static shared memory)
    cudaFuncAttributes fa;
    if (fp32) {
      CK(cudaFuncGetAttributes(&fa, k_mgpcg_persist<float>));
      if (psm + fa.sharedSizeBytes > (size_t)optin) return DROPLET_ERR_SIZE;
      CK(cudaFuncSetAttribute(k_mgpcg_persist<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes));
      // prefer L1 over shared memory beyond what a launch requests: the tail and the
      // tiles re-read the operator from L1
      CK(cudaFuncSetAttribute(k_mgpcg_persist<float>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxL1));
      pmg_smem_max = (size_t)(optin - (int)fa.sharedSizeBytes);
      CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mgpcg_persist<float>, PTPB, psm));
    } else {
      CK(cudaFuncGetAttributes(&fa, k_mgpcg_persist<double>));
      if (psm + fa.sharedSizeBytes > (size_t)optin) return DROPLET_ERR_SIZE;
      CK(cudaFuncSetAttribute(k_mgpcg_persist<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes));
      CK(cudaFuncSetAttribute(k_mgpcg_persist<double>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxL1));
      pmg_smem_max = (size_t)(optin - (int)fa.sharedSizeBytes);
      CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mgpcg_persist<double>, PTPB, psm));
    }
    pmg_blocks = per * nsm;
    nsm_ = nsm;
    if (pmg_blocks < 1) return DROPLET_ERR_SIZE;
  }
  mg_fp32 = fp32;
  mg_m[0] = mm[0]; mg_m[1] = mm[1]; mg_m[2] = mm[2];
  return 0;
}

int Solver::build_mg(const BoxSys& s, int fp32) {
  int rc = prepare_mg(s.m, fp32);
  if (rc) return rc;
  {   // the launched V-cycle's levels above its tail use the colour-ordered b and 1/diag
    int lt = nlev - 1;
    while (lt > 0 && lev[lt - 1].N <= TAIL_MAX_CELLS) --lt;
    for (int l = 0; l < nlev; ++l) lev[l].split = l < lt ? 1 : 0;
  }
  // level 0 operator: the pressure box in the hierarchy precision
  MGLevel& L0 = lev[0];
  int g0 = lin_grid(L0.N);
  if (fp32) {
    ++g_launches, k_cast<float, double><<<g0, TPB, 0, stream>>>(L0.N, (float*)L0.D, s.D);
    for (int a = 0; a < 3; ++a)
      if (L0.c[a]) ++g_launches, k_cast<float, double><<<g0, TPB, 0, stream>>>(L0.N, (float*)L0.c[a], s.c[a]);
  } else {
    // FP64 hierarchy: level 0 is the pressure box itself
    L0.D = s.D;
    for (int a = 0; a < 3; ++a) L0.c[a] = s.c[a];
  }
  for (int l = 1; l < nlev; ++l) {
    int gl = lin_grid(lev[l].N);
    if (fp32) {
      LevV<float> F = lv<float>(lev[l - 1]), C = lv<float>(lev[l]);
      ++g_launches, k_mg_coarsen<float><<<gl, TPB, 0, stream>>>(F, C, (float*)lev[l].D, (float*)lev[l].c[0], (float*)lev[l].c[1], (float*)lev[l].c[2]);
    } else {
      LevV<double> F = lv<double>(lev[l - 1]), C = lv<double>(lev[l]);
      ++g_launches, k_mg_coarsen<double><<<gl, TPB, 0, stream>>>(F, C, (double*)lev[l].D, (double*)lev[l].c[0], (double*)lev[l].c[1], (double*)lev[l].c[2]);
    }
  }
  for (int l = 0; l < nlev; ++l) {
    int gl = lin_grid(lev[l].N);
    if (fp32) ++g_launches, k_mg_idg<float><<<gl, TPB, 0, stream>>>(lv<float>(lev[l]), (float*)lev[l].idg);
    else ++g_launches, k_mg_idg<double><<<gl, TPB, 0, stream>>>(lv<double>(lev[l]), (double*)lev[l].idg);
  }
  CK(cudaGetLastError());
  return 0;
}

template <typename T>
static void smooth(Prof* prof, LevV<T> L, int col, int first, const int* done, cudaStream_t st) {
  int d = L.c[2] ? 3 : 2;
  ProfScope ps(prof, KC_MG_SMOOTH, st, (2.5 + d) * L.N * (double)sizeof(T),
               sizeof(T) == 8 ? (2.0 * d + 1.0) * 0.5 * L.N : 0.0);
  const long long n = half_sweep_threads(L.m);
  ++g_launches;
  if (n >= SWEEP_PAIR_MIN) {
    if (L.split) k_mg_smooth<T, true, 2><<<lin_grid((n + 1) / 2), TPB, 0, st>>>(L, col, first, done);
    else k_mg_smooth<T, false, 2><<<lin_grid((n + 1) / 2), TPB, 0, st>>>(L, col, first, done);
  } else {
    if (L.split) k_mg_smooth<T, true, 1><<<lin_grid(n), TPB, 0, st>>>(L, col, first, done);
    else k_mg_smooth<T, false, 1><<<lin_grid(n), TPB, 0, st>>>(L, col, first, done);
  }
}

// (ad0: the total diagonal of level 0 when it is the FP64 box whose CG formed it, else null)
template <typename T>
static void vcycle_t(Prof* prof, MGLevel* lev, int nlev, const int* done, cudaStream_t st, const T* ad0 = nullptr) {
  const int nu = 2;          // smoothing sweeps (red + black) before and after
  const int ncoarse = 4;     // symmetric sweep pairs on the coarsest level (at most 2^d x ... cells)
  // levels from `lt` on run inside one block (k_mg_tail)
  int lt = nlev - 1;
  while (lt > 0 && lev[lt - 1].N <= TAIL_MAX_CELLS) --lt;
  for (int l = 0; l < lt; ++l) {
    LevV<T> L = lv<T>(lev[l]);
    for (int s = 0; s < nu; ++s) {
      smooth<T>(prof, L, 0, s == 0, done, st);
      smooth<T>(prof, L, 1, 0, done, st);
    }
    LevV<T> C = lv<T>(lev[l + 1]);
    {
      int d = L.c[2] ? 3 : 2;
      const T* ad = l == 0 ? ad0 : nullptr;
      ProfScope ps(prof, KC_MG_RESTRICT, st, ((3.0 + d) * L.N + C.N) * (double)sizeof(T),
                   sizeof(T) == 8 ? (ad ? 2.0 * d + 2.0 : 4.0 * d + 3.0) * L.N : 0.0);
      ++g_launches, k_mg_restrict<T><<<lin_grid(C.N), TPB, 0, st>>>(L, C, done, ad);
    }
  }
  TailLevels<T> TL;
  for (int l = 0; l < nlev; ++l) TL.L[l] = lv<T>(lev[l]);
  TL.total = (int)tail_layout(lev, lt, nlev, sizeof(T), TL.xo, TL.bo);
  const size_t smem = (size_t)TL.total * sizeof(T);
  {
    // algorithmic bytes: the tail levels' operators (D, couplings, 1/diag) and the first
    // tail level's b in, its x out
    double tb = 2.0 * lev[lt].N;
    for (int l = lt; l < nlev; ++l) tb += (2.0 + (lev[l].c[2] ? 3 : 2)) * lev[l].N;
    ProfScope ps(prof, KC_MG_SMOOTH, st, tb * sizeof(T));
    ++g_launches, k_mg_tail<T><<<1, TAIL_THREADS, smem, st>>>(TL, lt, nlev, nu, ncoarse, done);
  }
  for (int l = lt - 1; l >= 0; --l) {
    LevV<T> L = lv<T>(lev[l]), C = lv<T>(lev[l + 1]);
    if constexpr (sizeof(T) == 4) {
      {
        // the prolongation inside the first colour-1 half sweep: the half sweep's bytes and
        // the coarse level's x
        const int d = L.c[2] ? 3 : 2;
        ProfScope ps(prof, KC_MG_SMOOTH, st, ((2.5 + d) * L.N + C.N) * (double)sizeof(T));
        const long long n = half_sweep_threads(L.m);
        ++g_launches;
        if (n >= SWEEP_PAIR_MIN) {
          if (L.split) k_mg_prolong_smooth<T, true, 2><<<lin_grid((n + 1) / 2), TPB, 0, st>>>(L, C, done);
          else k_mg_prolong_smooth<T, false, 2><<<lin_grid((n + 1) / 2), TPB, 0, st>>>(L, C, done);
        } else {
          if (L.split) k_mg_prolong_smooth<T, true, 1><<<lin_grid(n), TPB, 0, st>>>(L, C, done);
          else k_mg_prolong_smooth<T, false, 1><<<lin_grid(n), TPB, 0, st>>>(L, C, done);
        }
      }
      smooth<T>(prof, L, 0, 0, done, st);
      for (int s = 1; s < nu; ++s) {
        smooth<T>(prof, L, 1, 0, done, st);
        smooth<T>(prof, L, 0, 0, done, st);
      }
    } else {
      int g = lin_grid(L.N);
      {
        ProfScope ps(prof, KC_MG_PROLONG, st, (2.0 * L.N + C.N) * (double)sizeof(T), 1.0 * L.N);
        ++g_launches, k_mg_prolong<T><<<g, TPB, 0, st>>>(L, C, done);
      }
      for (int s = 0; s < nu; ++s) {
        smooth<T>(prof, L, 1, 0, done, st);
        smooth<T>(prof, L, 0, 0, done, st);
      }
    }
  }
}

// z = M r by one V-cycle; in an FP32 hierarchy with casts = false the caller has rounded r
// into level 0's b and widens level 0's x into z itself (fused into its CG kernels)
void Solver::vcycle(int fp32, bool casts) {
  MGLevel& L0 = lev[0];
  int g0 = lin_grid(L0.N);
  if (fp32) {
    if (casts) ++g_launches, k_cast_done<float, double><<<g0, TPB, 0, stream>>>(L0.N, (float*)L0.b, r, done);
    vcycle_t<float>(prof, lev, nlev, done, stream);
    if (casts) ++g_launches, k_cast_done<double, float><<<g0, TPB, 0, stream>>>(L0.N, z, (const float*)L0.x, done);
  } else {
    // level 0 of an FP64 hierarchy is the CG's box: its total diagonal is adg
    vcycle_t<double>(prof, lev, nlev, done, stream, adg);
  }
}

template <typename T>
int Solver::pcg_mg_persist(const BoxSys& s, double rtol, int maxit, SolveStats* out) {
  constexpr bool f32 = sizeof(T) == 4;
  // the hierarchy is built inside the kernel; an FP64 hierarchy's level 0 is the box
  int rc = prepare_mg(s.m, f32);
  if (rc) return rc;
  if (!f32) {
    lev[0].D = (void*)s.D;
    for (int q = 0; q < 3; ++q) lev[0].c[q] = (void*)s.c[q];
  }
  BoxV A = view(s);
  MgArgs<T> a;
  memset(&a, 0, sizeof(a));
  a.A = A;
  a.b = s.b;
  a.tol2 = rtol * rtol;
  a.maxit = maxit;
  a.cast0 = f32;
  a.rec = take_record();
  a.x = s.x;
  a.r[0] = r;
  a.r[1] = z;
  a.q[0] = Ap;
  a.q[1] = mg_q2;
  a.p = p;
  a.w = idg;
  for (int l = 0; l < nlev; ++l) a.TL.L[l] = lv<T>(lev[l]);
  int lt = nlev - 1;
  while (lt > 0 && lev[lt - 1].N <= PMG_TAIL_MAX_CELLS) --lt;
  const int ldn = dense_level(lev, lt, nlev, f32);
  a.nlev = ldn >= 0 ? ldn + 1 : nlev;
  a.dn = ldn >= 0 ? (int)lev[ldn].N : 0;
  a.lt = lt;
  a.ncoarse = 4;
  a.z0 = (lt > 0 && lev[0].m[2] == 1) ? (const T*)lev[0].xp : (const T*)lev[0].x;
  a.TL.total = (int)tail_layout(lev, lt, a.nlev, sizeof(T), a.TL.xo, a.TL.bo);
  a.part = part;
  a.stat = sc;
  a.done = done;
  a.bar = bar;
  a.err = err;
  a.spin = spin_limit;
  a.tx = (mg_tile[0] + 1) & ~1;   // even: the fused restriction's aggregates stay in a tile
  a.ty = (mg_tile[1] + 1) & ~1;
  PmgLayout pl = pmg_layout(a.TL.total, sizeof(T), a.tx, a.ty, a.dn);
  if (pl.bytes > pmg_smem_max) {   // the chosen tile does not fit: the default one does
    a.tx = a.ty = 32;
    pl = pmg_layout(a.TL.total, sizeof(T), a.tx, a.ty, a.dn);
  }
  a.dw = pl.dw;
  a.dp = pl.dp;
  const size_t smem = pl.bytes;
  int grid = (int)((s.N + PTPB - 1) / PTPB);
  if (grid > pmg_blocks) grid = pmg_blocks;
  if (sm_budget > 0) grid = std::min(grid, sm_budget * std::max(1, pmg_blocks / nsm_));
  if (grid > RED_BLOCKS) grid = RED_BLOCKS;
  if (grid < 1) grid = 1;
  cudaLaunchConfig_t lc;
  memset(&lc, 0, sizeof(lc));
  lc.gridDim = dim3(grid);
  lc.blockDim = dim3(PTPB);
  lc.dynamicSmemBytes = smem;
  lc.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  // algorithmic bytes per iteration: level-0 FP64 vectors (update: x, r, p, q, w in,
  // x, r, p, q out; w = A z: operator in, w out), the level-0 b and z in the hierarchy
  // precision, each grid level's operator, b and x once per smoothing side and the
  // transfers, and the tail; binary64 instructions: the CG update (four FMAs, three dot
  // products) and w = A z (difference form), plus the sweeps of an FP64 hierarchy
  const double d = s.c[2] ? 3.0 : 2.0, es = (double)sizeof(T), N0 = (double)s.N;
  double iter_b = (9.0 * 8.0 + 3.0 * es) * N0 + ((1.0 + d) * 8.0 + 16.0 + es) * N0;
  double iter_f = (8.0 + 4.0 * d) * N0;
  for (int l = 0; l < lt; ++l) {
    const double Nl = (double)lev[l].N, Nc = (double)lev[l + 1].N;
    iter_b += 2.0 * (3.0 + d) * Nl * es + ((3.0 + d) * Nl + Nc) * es + (2.0 * Nl + Nc) * es;
    if (!f32) iter_f += 4.0 * MG_NU * (1.0 + 2.0 * d) * 0.5 * Nl;
  }
  iter_b += 2.0 * lev[lt].N * es;
  for (int l = lt; l < nlev; ++l) iter_b += (2.0 + d) * lev[l].N * es;
  ++g_launches;
  {
    ProfScope ps(prof, KC_MG_SMOOTH, stream, 0.0);
    CK(cudaLaunchKernelEx(&lc, k_mgpcg_persist<T>, a));
  }
  if (capturing) return 0;
  int conv = 0;
  poll(hsc, sc, done, stream, maxit, &conv);
  if (prof && prof->on) {
    prof->bytes[KC_MG_SMOOTH] += hsc[S_ITS] * iter_b;
    prof->flops[KC_MG_SMOOTH] += hsc[S_ITS] * iter_f;
  }
  fill_stats(hsc, conv, out);
  return persist_status(hsc, conv);
}

int Solver::pcg_mg(const BoxSys& s, double rtol, int maxit, int fp32, SolveStats* out) {
  if (persistent) return fp32 ? pcg_mg_persist<float>(s, rtol, maxit, out) : pcg_mg_persist<double>(s, rtol, maxit, out);
  int rc = build_mg(s, fp32);
  if (rc) return rc;
  if (!fp32) { lev[0].b = r; lev[0].x = z; }
  BoxV A = view(s);
  int nb = cg_grid(s.N);
  int g = lin_grid(s.N);
  ++g_launches, k_pcg_init<<<nb, TPB, 0, stream>>>(A, s.b, s.x, r, z, p, idg, 0, part, adg);
  ++g_launches, k_fin_init<<<1, TPB, 0, stream>>>(part, nb, sc, done, rtol * rtol, maxit, nullptr, nullptr);
  vcycle(fp32, true);
  ++g_launches, k_dot_rz<<<nb, TPB, 0, stream>>>(s.N, r, z, part, done, sc, cnt, 1);
  float* const bf = fp32 ? (float*)lev[0].b : nullptr;
  const float* const zf = fp32 ? (const float*)lev[0].x : nullptr;
  ++g_launches, k_cast_done<double, double><<<g, TPB, 0, stream>>>(s.N, p, z, done);
  auto iteration = [&]() {
    {
      ProfScope ps(prof, KC_SPMV, stream, (3.0 + (s.c[2] ? 3 : 2)) * s.N * 8.0, (2.0 * (s.c[2] ? 3 : 2) + 2.0) * s.N);
      ++g_launches, k_spmv_dot<<<nb, TPB, 0, stream>>>(A, p, Ap, part, done, sc, cnt, adg);
    }
    {
      ProfScope ps(prof, KC_UPDATE, stream, (6.0 * 8.0 + (fp32 ? 4.0 : 0.0)) * s.N, 3.0 * s.N);
      ++g_launches, k_update<<<nb, TPB, 0, stream>>>(s.N, s.x, r, p, Ap, idg, z, 0, sc, part, done, cnt, bf);
    }
    vcycle(fp32, false);
    ++g_launches, k_dot_rz<<<nb, TPB, 0, stream>>>(s.N, r, z, part, done, sc, cnt, 0, zf);
    ++g_launches, k_p_update<<<red_grid_cap(s.N, rb), TPB, 0, stream>>>(s.N, p, z, sc, done);
  };
  if (capturing) return device_loop(iteration);
  const int chunk = (prof && prof->on) ? 1 : 4;
  int conv = 0;
  for (int it = 0; it < maxit; it += chunk) {
    for (int q = 0; q < chunk; ++q) iteration();
    CK(cudaGetLastError());
    if (poll(hsc, sc, done, stream, maxit, &conv)) break;
  }
  if (!conv) poll(hsc, sc, done, stream, maxit, &conv);
  fill_stats(hsc, conv, out);
  return conv ? 0 : DROPLET_ERR_NOT_CONVERGED;
}

// ---------------------------------------------------------------- no-allocation box solve
// Work vectors of droplet_box_solve_noalloc: r, z, p, Ap, 1/diag (5 x max unknowns),
// reduction partials, CG scalars and the done flag, in one static device array.
constexpr long long NA_MAX = DROPLET_NOALLOC_MAX_UNKNOWNS;
constexpr long long NA_PART = (long long)RED_BLOCKS * 8;
constexpr long long NA_WORDS = 5 * NA_MAX + NA_PART + S_COUNT + 8;
static __device__ __align__(256) double g_noalloc_ws[NA_WORDS];

// Device address of the array in the current device's context.  Host code may not use
// the symbol itself (it names a host-side stand-in), so every call looks the address up
// again: the lookup allocates nothing, and a cached address would go stale when the
// context is replaced (cudaDeviceReset, or a caller that switches driver contexts).
static int noalloc_workspace(double** out) {
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_ws);
  if (e != cudaSuccess || !ptr) {
    fprintf(stderr, "droplet: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
    return DROPLET_ERR_CUDA;
  }
  *out = (double*)ptr;
  return 0;
}

}  // namespace dg

extern "C" int droplet_box_solve_noalloc(const int m[3], const double* D, const double* c0, const double* c1,
                                         const double* c2, const double* b, double* x, double rtol, int maxit,
                                         void* cuda_stream, int* its, double* relres) {
  using namespace dg;
  if (!m || !D || !c0 || !c1 || !b || !x || maxit < 1 || !(rtol > 0.0)) return DROPLET_ERR_ARG;
  if (m[0] < 1 || m[1] < 1 || m[2] < 1 || (m[2] > 1 && !c2)) return DROPLET_ERR_ARG;
  // every dimension is at least 1, so one above the limit already exceeds it (and the
  // product below cannot wrap)
  if (m[0] > NA_MAX || m[1] > NA_MAX || m[2] > NA_MAX) {
    fprintf(stderr, "droplet_box_solve_noalloc: a box dimension exceeds the static workspace (%lld)\n", NA_MAX);
    return DROPLET_ERR_SIZE;
  }
  long long N = (long long)m[0] * m[1] * m[2];
  if (N > NA_MAX) {
    fprintf(stderr, "droplet_box_solve_noalloc: %lld unknowns exceed the static workspace (%lld)\n", N, NA_MAX);
    return DROPLET_ERR_SIZE;
  }
  // the call reads the solver's state back and synchronises its stream, which no stream
  // capture allows: refused before anything is enqueued
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing((cudaStream_t)cuda_stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    fprintf(stderr, "droplet_box_solve_noalloc: the stream is being captured\n");
    return DROPLET_ERR_ARG;
  }
  double* ws = nullptr;
  int rc = noalloc_workspace(&ws);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double *r = ws, *z = ws + NA_MAX, *p = ws + 2 * NA_MAX, *Ap = ws + 3 * NA_MAX, *idg = ws + 4 * NA_MAX;
  double* part = ws + 5 * NA_MAX;
  double* sc = part + NA_PART;
  int* done = (int*)(sc + S_COUNT);
  BoxV A;
  for (int a = 0; a < 3; ++a) A.m[a] = m[a];
  A.N = N;
  A.D = D;
  A.c[0] = c0;
  A.c[1] = c1;
  A.c[2] = m[2] > 1 ? c2 : nullptr;
  int nb = red_grid(N);
  // every vector, partial, scalar and the flag are written by k_pcg_init / k_fin_init before use
  k_pcg_init<<<nb, TPB, 0, st>>>(A, b, x, r, z, p, idg, 1, part);
  k_fin_init<<<1, TPB, 0, st>>>(part, nb, sc, done, rtol * rtol, maxit, nullptr, nullptr);
  double hs[S_COUNT + 1];
  int d = 0;
  for (int it = 0; it < maxit; it += 8) {
    for (int q = 0; q < 8; ++q) {
      k_spmv_dot<<<nb, TPB, 0, st>>>(A, p, Ap, part, done, sc, nullptr);
      k_fin_alpha<<<1, TPB, 0, st>>>(part, nb, sc, done);
      k_update<<<nb, TPB, 0, st>>>(N, x, r, p, Ap, idg, z, 1, sc, part, done, nullptr);
      k_fin_iter<<<1, TPB, 0, st>>>(part, nb, sc, done, 1);
      k_p_update<<<nb, TPB, 0, st>>>(N, p, z, sc, done);
    }
    if (cudaGetLastError() != cudaSuccess) return DROPLET_ERR_CUDA;
    // pageable host destination: no pinned allocation
    if (cudaMemcpyAsync(hs, sc, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&d, done, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return DROPLET_ERR_CUDA;
    if (d != 0) break;
  }
  if (its) *its = (int)hs[S_ITS];
  if (relres) *relres = hs[S_BB] > 0 ? sqrt(hs[S_RR] / hs[S_BB]) : 0.0;
  return d == 1 ? 0 : DROPLET_ERR_NOT_CONVERGED;
}
