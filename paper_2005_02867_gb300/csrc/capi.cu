// C ABI of the droplet library (include/droplet.h): context lifetime, the
// per-step stage sequence of Sec. 3.1 (Fig. Scheme), diagnostics and field
// access.  Every stage runs in the kernels of step_kernels.cu and solver.cu;
// this file only allocates, launches and copies.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>
#include <algorithm>
#include <cmath>
#include "kernels.h"

using namespace dg;

#define CKR(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { fprintf(stderr, "droplet: %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); return DROPLET_ERR_CUDA; } } while (0)

struct dctx {
  cudaStream_t st = nullptr;
  droplet_config cfg;
  Geo g;
  Phys p;
  // state
  double *alpha = nullptr, *T = nullptr, *omega = nullptr, *pr = nullptr, *rhoG = nullptr, *u[3] = {nullptr, nullptr, nullptr};
  // step work arrays
  double *rhoG_old = nullptr, *mdot = nullptr, *mraw = nullptr, *astar = nullptr, *aL = nullptr, *Rp = nullptr, *Rm = nullptr;
  float* astar_f = nullptr;          // alpha* in binary32 for the face stencils (mixed precision)
  Shadow32 s32{};                    // binary32 copies for the assembly stencils (mixed precision)
  double *FL[3] = {nullptr, nullptr, nullptr}, *AF[3] = {nullptr, nullptr, nullptr}, *us[3] = {nullptr, nullptr, nullptr};
  double *xi = nullptr;
  // history of the Helmholtz unknowns (previous step's T, omega, face velocities) for the
  // extrapolated initial guesses; valid while scal[SC_HIST] = 1
  double *hT = nullptr, *hW = nullptr, *hu[3] = {nullptr, nullptr, nullptr};
  double *rho = nullptr, *mu = nullptr, *kc = nullptr, *cp = nullptr, *Dm = nullptr, *yq = nullptr, *dp = nullptr, *S = nullptr;
  int* adj = nullptr;
  unsigned char* solid = nullptr;    // the fibre's cells (droplet_config.fiber = 1), else null
  double *bD = nullptr, *bc[3] = {nullptr, nullptr, nullptr}, *brhs = nullptr, *bx = nullptr;
  // box systems (D, c0, c1, c2, rhs, x each) of the joint momentum solve: of the second and
  // third velocity component (the first uses the shared box), or of every component when
  // the momentum stage runs on its own branch
  double* xb[3][6] = {{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr},
                      {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr},
                      {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr}};
  double *part = nullptr, *psum = nullptr, *pmax = nullptr, *scal = nullptr;
  // the liquid's expansion term of the last continuity source (a temperature-dependent
  // liquid density only, else null): the next alpha source subtracts it
  double* expand = nullptr;
  unsigned* flags = nullptr;
  int* dirty = nullptr;              // a state field was overwritten: S0 re-evaluates rho_G everywhere
  double* hscal = nullptr;
  unsigned* hflags = nullptr;
  Solver solver;
  // the momentum stage of a single droplet on a branch of its own, concurrent with energy
  // and species: its solver workspace, stream and fork / join events
  bool conc = false;
  Solver solver_m;
  cudaStream_t stm = nullptr;
  cudaEvent_t evf = nullptr, evj = nullptr;
  Prof prof;
  cudaStream_t st2 = nullptr;        // capture stream of the solver loop bodies
  cudaStream_t own = nullptr;        // the droplet's own stream in a batch
  int rb = RED_BLOCKS;               // block cap of the reduction kernels
  int its_p = 0, its_T = 0, its_w = 0, its_u = 0;
  double res_p = 0.0, t = 0.0;
  long long step = 0;
};

static const char* kErr[] = {"ok", "invalid argument", "CUDA error", "linear solve not converged",
                             "non-finite value", "buffer size mismatch", "device allocation failed",
                             "checkpoint file error", "device wait timed out"};

extern "C" const char* droplet_strerror(int s) {
  if (s > 0 || s < -8) return "unknown status";
  return kErr[-s];
}

// A solve that reached its cap (NOT_CONVERGED) or whose grid-barrier wait ran out
// (TIMEOUT) leaves the step running: the mark goes to *nc (1 = not converged, 2 = timed
// out, the larger kept) and 0 is returned; any other error is returned as it is.
static int soft_status(int rc, int* nc) {
  if (rc == DROPLET_ERR_NOT_CONVERGED) { if (*nc < 1) *nc = 1; return 0; }
  if (rc == DROPLET_ERR_TIMEOUT) { *nc = 2; return 0; }
  return rc;
}

static int check_cfg(const droplet_config& c) {
  if (c.geom != 0 && c.geom != 1) return DROPLET_ERR_ARG;
  int na = c.geom == 0 ? 2 : 3;
  for (int a = 0; a < na; ++a) {
    if (c.n[a] < 4 || c.n[a] > 16384 || !(c.L[a] > 0.0)) return DROPLET_ERR_ARG;
  }
  if (!(c.dt > 0.0) || !(c.D0 > 0.0) || !(c.P > 0.0) || !(c.T_amb > 0.0) || !(c.T_drop > 0.0)) return DROPLET_ERR_ARG;
  for (int a = 0; a < na; ++a)
    if (c.xc[a] < 0.0 || c.xc[a] > c.L[a]) return DROPLET_ERR_ARG;
  if (c.geom == 0 && c.xc[0] != 0.0) return DROPLET_ERR_ARG;
  if (c.eq_model != 0 && c.eq_model != 1) return DROPLET_ERR_ARG;
  if (c.bc_mode != 0 && c.bc_mode != 1) return DROPLET_ERR_ARG;
  if (c.cg_maxit < 1 || c.helm_maxit < 1 || !(c.cg_rtol > 0.0) || !(c.helm_rtol > 0.0)) return DROPLET_ERR_ARG;
  if (c.precision != 0 && c.precision != 1) return DROPLET_ERR_ARG;
  for (int a = 0; a < 2; ++a)
    if (c.mg_tile[a] != 0 && (c.mg_tile[a] < 8 || c.mg_tile[a] > 256)) return DROPLET_ERR_ARG;
  if (c.wait_limit < 0 || (c.solver_select != 0 && c.solver_select != 1)) return DROPLET_ERR_ARG;
  if (!(c.co_max >= 0.0) || !std::isfinite(c.co_max)) return DROPLET_ERR_ARG;
  if (c.adv_scheme != 0 && c.adv_scheme != 1) return DROPLET_ERR_ARG;
  // the fibre: the compressive advection, a constant liquid density
  if (c.fiber != 0 && c.fiber != 1) return DROPLET_ERR_ARG;
  if (c.fiber == 1 && (c.adv_scheme != 0 || c.drho_l_dT != 0.0 || !(c.fiber_radius > 0.0)))
    return DROPLET_ERR_ARG;
  // a liquid density linear in T stays positive up to the ambient and boiling temperatures
  if (!std::isfinite(c.drho_l_dT) || !(c.rho_l + c.drho_l_dT * (c.T_amb - c.T_drop) > 0.0) ||
      !(c.rho_l + c.drho_l_dT * (c.Tb - c.T_drop) > 0.0))
    return DROPLET_ERR_ARG;
  long long nn = (long long)c.n[0] * c.n[1] * (c.geom == 0 ? 1 : c.n[2]);
  {   // 32-bit cell and face indices: the cells plus the largest extra face plane
    const long long n2 = c.geom == 0 ? 1 : c.n[2];
    const long long plane = std::max((long long)c.n[0] * c.n[1], std::max((long long)c.n[1] * n2, (long long)c.n[0] * n2));
    if (nn + plane >= (1LL << 31)) return DROPLET_ERR_ARG;
  }
  return 0;
}

// Products rounded on their own (no fused multiply-add on any host), so that the fibre's
// cells below are those of the same formula evaluated operation by operation.
static __attribute__((noinline)) double mul_rounded(double a, double b) { return a * b; }

// The fibre's solid cells (Sec. 3.1.1, Table tableboundary "sphere" row): the cells whose
// centre lies closer than fiber_radius to the droplet centre,
// sqrt(sum over the active axes of ((i_a + 1/2) h_a - xc_a)^2) < fiber_radius.
static void fibre_cells(const Geo& g, const droplet_config& c, std::vector<unsigned char>& m) {
  m.assign((size_t)g.N, 0);
  const int na = nact(g);
  for (int k = 0; k < g.n[2]; ++k)
    for (int j = 0; j < g.n[1]; ++j)
      for (int i = 0; i < g.n[0]; ++i) {
        const int q[3] = {i, j, k};
        double d2 = 0.0;
        for (int a = 0; a < na; ++a) {
          const double t = mul_rounded(q[a] + 0.5, g.h[a]) - c.xc[a];
          d2 = d2 + mul_rounded(t, t);
        }
        m[(size_t)i + (size_t)g.n[0] * ((size_t)j + (size_t)g.n[1] * k)] = std::sqrt(d2) < c.fiber_radius ? 1 : 0;
      }
}

static void make_geo(const droplet_config& c, Geo& g) {
  memset(&g, 0, sizeof(g));
  g.axisym = c.geom == 0;
  g.act3 = !g.axisym;
  g.n[0] = c.n[0];
  g.n[1] = c.n[1];
  g.n[2] = g.axisym ? 1 : c.n[2];
  for (int a = 0; a < 3; ++a) g.h[a] = (a < 2 || !g.axisym) ? c.L[a] / g.n[a] : 1.0;
  for (int a = 0; a < 3; ++a) g.ih[a] = 1.0 / g.h[a];
  g.hmin = g.axisym ? fmin(g.h[0], g.h[1]) : fmin(g.h[0], fmin(g.h[1], g.h[2]));
  g.vol3 = g.h[0] * g.h[1] * g.h[2];
  for (int a = 0; a < 3; ++a) g.area3[a] = g.vol3 * g.ih[a];
  g.gthr = 1e-8 / g.hmin;
  g.hvol3 = 0.5 * g.vol3;
  for (int a = 0; a < 3; ++a) {
    g.aih[a] = g.area3[a] * g.ih[a];
    g.aih2[a] = 2.0 * g.aih[a];
    g.qaih[a] = 0.25 * g.aih[a];
    g.qih[a] = 0.25 * g.ih[a];
    for (int b = 0; b < 3; ++b) g.qvt[b][a] = 0.25 * g.area3[a] * g.ih[b];
  }
  {
    const int na = g.axisym ? 2 : 3;
    for (int a = 0; a < na; ++a) {
      g.gh[a] = c.g[a] * g.h[a];
      if (c.g[a] != 0.0) g.gmask |= 1 << a;
    }
    for (int b = 0; b < na; ++b)
      for (int a = 0; a < na; ++a)
        if (a != b && (g.gmask >> a & 1)) g.gxc[b] += 0.5 * g.gh[a];
  }
  g.s = g.axisym ? 1 : 2;
  int inlet = c.bc_mode == 1 ? BC_FORCED : BC_OPEN;
  if (g.axisym) {
    g.bc[0][0] = BC_AXIS; g.bc[0][1] = BC_WALL;
    g.bc[1][0] = inlet;   g.bc[1][1] = BC_OPEN;
    g.bc[2][0] = BC_WALL; g.bc[2][1] = BC_WALL;
  } else {
    g.bc[0][0] = BC_WALL; g.bc[0][1] = BC_WALL;
    g.bc[1][0] = BC_WALL; g.bc[1][1] = BC_WALL;
    g.bc[2][0] = inlet;   g.bc[2][1] = BC_OPEN;
  }
  g.N = (long long)g.n[0] * g.n[1] * g.n[2];
}

static void make_phys(const droplet_config& c, Phys& p) {
  memset(&p, 0, sizeof(p));
  p.D0 = c.D0; p.T_drop = c.T_drop; p.T_amb = c.T_amb; p.P = c.P;
  for (int a = 0; a < 3; ++a) { p.g[a] = c.g[a]; p.xc[a] = c.xc[a]; }
  if (c.geom == 0) p.g[2] = 0.0;
  p.u_in = c.u_inflow;
  p.Tb = c.Tb; p.Lv = c.Lv; p.M_l = c.M_l; p.rho_l = c.rho_l; p.cp_l = c.cp_l; p.k_l = c.k_l; p.mu_l = c.mu_l; p.D_l = c.D_l;
  p.M_g = c.M_g; p.cp_g = c.cp_g; p.cp_v = c.cp_v; p.k_g = c.k_g; p.mu_g = c.mu_g; p.D_g = c.D_g;
  p.Tc = c.Tc; p.Pc = c.Pc; p.om = c.omega_ac; p.Tc_g = c.Tc_g; p.Pc_g = c.Pc_g; p.om_g = c.omega_g; p.kij = c.kij;
  p.xi0 = c.xi0; p.Df = c.fiber_radius; p.dt = c.dt; p.C_alpha = c.C_alpha; p.T_perturb = c.T_perturb;
  p.idt = 1.0 / c.dt;
  p.dyn = nullptr;            // set once the device scalars exist (adaptive runs)
  p.co_hmin = 0.0;
  p.D_gas = c.D_g * (1.0e5 / c.P);
  p.rhoG_const = c.P * c.M_g / (R_GAS * c.T_amb);
  p.seed = c.seed;
  p.eq_model = c.eq_model;
  p.const_props = c.const_props_check;
  p.physics = c.physics_mask;
  const double Tc[2] = {c.Tc, c.Tc_g}, Pc[2] = {c.Pc, c.Pc_g}, om[2] = {c.omega_ac, c.omega_g};
  for (int s = 0; s < 2; ++s) {
    p.pr_ac[s] = 0.45724 * R_GAS * R_GAS * Tc[s] * Tc[s] / Pc[s];
    p.pr_b[s] = 0.07780 * R_GAS * Tc[s] / Pc[s];
    p.pr_k[s] = 0.37464 + 1.54226 * om[s] - 0.26992 * om[s] * om[s];
    p.pr_siTc[s] = sqrt(1.0 / Tc[s]);
  }
  p.pr_sqac01 = std::sqrt(p.pr_ac[0] * p.pr_ac[1]) * (1.0 - c.kij);
  p.iM_l = 1.0 / c.M_l;
  p.iM_g = 1.0 / c.M_g;
  p.cc_LMR = c.Lv * c.M_l / R_GAS;
  p.iTb = 1.0 / c.Tb;
  p.irho_l = 1.0 / c.rho_l;
  p.drl = c.drho_l_dT;
}

static int dalloc(double** q, long long n) {
  if (cudaMalloc((void**)q, sizeof(double) * (size_t)(n > 0 ? n : 1)) != cudaSuccess) return DROPLET_ERR_NOMEM;
  return 0;
}

static void free_all(dctx* c) {
  double** arrs[] = {&c->alpha, &c->T, &c->omega, &c->pr, &c->rhoG, &c->rhoG_old, &c->mdot, &c->mraw, &c->astar,
                     &c->aL, &c->Rp, &c->Rm, &c->rho, &c->mu, &c->kc, &c->cp, &c->Dm, &c->yq, &c->dp, &c->S,
                     &c->bD, &c->brhs, &c->bx, &c->part, &c->psum, &c->pmax, &c->scal, &c->xi, &c->hT, &c->hW,
                     &c->expand};
  for (auto q : arrs) { cudaFree(*q); *q = nullptr; }
  for (int a = 0; a < 3; ++a) {
    cudaFree(c->u[a]); cudaFree(c->FL[a]); cudaFree(c->AF[a]); cudaFree(c->us[a]); cudaFree(c->bc[a]); cudaFree(c->hu[a]);
    c->u[a] = c->FL[a] = c->AF[a] = c->us[a] = c->bc[a] = c->hu[a] = nullptr;
  }
  for (auto& set : c->xb)
    for (auto& q : set) { cudaFree(q); q = nullptr; }
  cudaFree(c->adj); cudaFree(c->flags); cudaFree(c->dirty); cudaFree(c->astar_f); cudaFree(c->solid);
  c->adj = nullptr; c->flags = nullptr; c->dirty = nullptr; c->astar_f = nullptr; c->solid = nullptr;
  {
    float** sh[] = {&c->s32.T, &c->s32.w, &c->s32.k, &c->s32.gD, &c->s32.mu, &c->s32.u[0], &c->s32.u[1], &c->s32.u[2]};
    for (auto q : sh) { cudaFree(*q); *q = nullptr; }
  }
  cudaFreeHost(c->hscal); cudaFreeHost(c->hflags);
  c->hscal = nullptr; c->hflags = nullptr;
  c->solver.release();
  c->solver_m.release();
  if (c->evf) cudaEventDestroy(c->evf);
  if (c->evj) cudaEventDestroy(c->evj);
  if (c->stm) cudaStreamDestroy(c->stm);
  c->evf = c->evj = nullptr;
  c->stm = nullptr;
  c->prof.destroy();
  if (c->st2) cudaStreamDestroy(c->st2);
  if (c->own) cudaStreamDestroy(c->own);
  c->st2 = nullptr; c->own = nullptr;
}

// diagnostics of the current state; mode (DIAG_*): the end of a step (the history fields
// then hold the step's starting values; the clock advances and an adaptive run takes its
// next dt), an initial state (an adaptive run takes its first dt), or a state set from
// outside (history marked invalid, clock and dt kept)
static int run_diag(dctx* c, int mode) {
  Geo& g = c->g;
  int nb = red_grid_cap(g.N, c->rb);
  L_diag(c->st, nb, g, c->p, c->alpha, c->T, c->mdot, c->omega, c->rhoG, c->u[0], c->u[1], c->u[2] ? c->u[2] : c->u[0],
                                c->psum, c->pmax, c->flags);
  ++g_launches, k_diag_finish<<<1, TPB, 0, c->st>>>(c->psum, c->pmax, nb, c->scal, mode, c->p.co_hmin, c->cfg.dt);
  CKR(cudaGetLastError());
  return 0;
}

// The clock at t = 0 with the configured dt (the first step of an adaptive run then takes
// its dt from the initial velocities, DIAG_INITIAL); enqueued on st.
static void reset_clock(dctx* c, cudaStream_t st) {
  const double v[3] = {c->cfg.dt, 1.0 / c->cfg.dt, 0.0};   // SC_DT, SC_IDT, SC_TIME
  cudaMemcpyAsync(c->scal + SC_DT, v, sizeof(v), cudaMemcpyHostToDevice, st);
}

// One droplet's context: device memory, solver workspace and the initial state (Sec. 3.3).
// own_stream: the droplet works on a stream of its own (a branch of the batch graph).
static int init_one(const droplet_config& cfg, cudaStream_t main_st, bool own_stream, dctx** out) {
  *out = nullptr;
  int rc;
  dctx* c = new (std::nothrow) dctx();
  if (!c) return DROPLET_ERR_NOMEM;
  c->cfg = cfg;
  c->st = main_st;
  if (own_stream) {
    if (cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking) != cudaSuccess) { delete c; return DROPLET_ERR_CUDA; }
    c->st = c->own;
  }
  if (cudaStreamCreateWithFlags(&c->st2, cudaStreamNonBlocking) != cudaSuccess) { free_all(c); delete c; return DROPLET_ERR_CUDA; }
  make_geo(c->cfg, c->g);
  make_phys(c->cfg, c->p);
  Geo& g = c->g;
  long long N = g.N;
  int na = nact(g);
  double** cells[] = {&c->alpha, &c->T, &c->omega, &c->pr, &c->rhoG, &c->rhoG_old, &c->mdot, &c->mraw, &c->astar,
                      &c->aL, &c->Rp, &c->Rm, &c->rho, &c->mu, &c->kc, &c->cp, &c->Dm, &c->yq, &c->dp, &c->S,
                      &c->bD, &c->brhs, &c->bx, &c->xi, &c->hT, &c->hW};
  for (auto q : cells)
    if ((rc = dalloc(q, N))) { free_all(c); delete c; return rc; }
  if (c->cfg.precision == 1) {
    bool ok = cudaMalloc((void**)&c->astar_f, sizeof(float) * (size_t)N) == cudaSuccess;
    float** sh[] = {&c->s32.T, &c->s32.w, &c->s32.k, &c->s32.gD, &c->s32.mu};
    for (auto q : sh) ok = ok && cudaMalloc((void**)q, sizeof(float) * (size_t)N) == cudaSuccess;
    for (int a = 0; a < na; ++a)
      ok = ok && cudaMalloc((void**)&c->s32.u[a], sizeof(float) * (size_t)nfaces(g, a)) == cudaSuccess;
    if (!ok) { free_all(c); delete c; return DROPLET_ERR_NOMEM; }
  }

  for (int a = 0; a < 3; ++a) {
    if ((rc = dalloc(&c->bc[a], N))) { free_all(c); delete c; return rc; }
    if (a >= na) continue;
    long long nf = nfaces(g, a);
    if ((rc = dalloc(&c->u[a], nf)) || (rc = dalloc(&c->FL[a], nf)) || (rc = dalloc(&c->AF[a], nf)) ||
        (rc = dalloc(&c->us[a], nf)) || (rc = dalloc(&c->hu[a], nf))) { free_all(c); delete c; return rc; }
  }
  if ((rc = dalloc(&c->part, RED_BLOCKS * 8)) || (rc = dalloc(&c->psum, RED_BLOCKS * 7)) ||
      (rc = dalloc(&c->pmax, RED_BLOCKS * 3)) || (rc = dalloc(&c->scal, SC_COUNT))) { free_all(c); delete c; return rc; }
  if (cudaMalloc((void**)&c->adj, sizeof(int) * N) != cudaSuccess || cudaMalloc((void**)&c->flags, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc((void**)&c->dirty, sizeof(int)) != cudaSuccess ||
      cudaMallocHost((void**)&c->hscal, sizeof(double) * SC_COUNT) != cudaSuccess ||
      cudaMallocHost((void**)&c->hflags, sizeof(unsigned)) != cudaSuccess) { free_all(c); delete c; return DROPLET_ERR_NOMEM; }
  if (cfg.fiber == 1) {
    std::vector<unsigned char> m;
    fibre_cells(g, cfg, m);
    if (cudaMalloc((void**)&c->solid, (size_t)N) != cudaSuccess) { free_all(c); delete c; return DROPLET_ERR_NOMEM; }
    if (cudaMemcpy(c->solid, m.data(), (size_t)N, cudaMemcpyHostToDevice) != cudaSuccess) {
      free_all(c);
      delete c;
      return DROPLET_ERR_CUDA;
    }
    g.fib = 1;
    g.solid = c->solid;
    // the box of the solid cells (an empty mask gives an empty box: lo > hi)
    for (int a = 0; a < 3; ++a) { g.fib_lo[a] = g.n[a]; g.fib_hi[a] = -1; }
    for (int k = 0; k < g.n[2]; ++k)
      for (int j = 0; j < g.n[1]; ++j)
        for (int i = 0; i < g.n[0]; ++i)
          if (m[(size_t)i + (size_t)g.n[0] * ((size_t)j + (size_t)g.n[1] * k)]) {
            const int q[3] = {i, j, k};
            for (int a = 0; a < 3; ++a) {
              g.fib_lo[a] = std::min(g.fib_lo[a], q[a]);
              g.fib_hi[a] = std::max(g.fib_hi[a], q[a]);
            }
          }
    // no cell centre inside the sphere (a fibre finer than the grid): nothing is solid, and the
    // kernels run without the fibre's tests (whose box test needs a non-empty box)
    if (g.fib_hi[0] < 0) {
      g.fib = 0;
      g.solid = nullptr;
    }
  }
  c->solver.f32_helm = c->cfg.precision == 1;
  // latency-bound sizes: persistent solvers (in a batch each droplet is later given an
  // SM budget so that the cooperative solves of all branches fit the GPU together)
  c->solver.persistent = N <= Solver::PERSIST_MAX_CELLS;
  c->solver.persist_pcg = N <= (c->solver.f32_helm ? Solver::PERSIST_PCG_MAX_CELLS : Solver::PERSIST_MAX_CELLS);
  if (cfg.solver_select == 1) c->solver.persistent = c->solver.persist_pcg = false;   // launched solvers at any size
  if (cfg.wait_limit > 0) c->solver.spin_limit = cfg.wait_limit;
  // the velocity components are solved together (one persistent launch)
  const bool joint = c->solver.persist_pcg && (cfg.physics_mask & DROPLET_PHYS_FLOW);
  c->solver.nsys_extra = joint ? nact(c->g) - 1 : 0;
  // a single droplet whose solves all run persistently forks the momentum stage (S7) onto a
  // branch of its own, concurrent with energy and species (S5, S6): neither reads what the
  // other writes, and both latency-bound chains then share the GPU
  c->conc = joint && !own_stream && c->solver.persistent;
  const int nsets = c->conc ? na : c->solver.nsys_extra;
  for (int k = 0; k < nsets; ++k)
    for (int q = 0; q < 6; ++q)
      if (q != 3 || na == 3)
        if ((rc = dalloc(&c->xb[k][q], N))) { free_all(c); delete c; return rc; }
  if (cfg.mg_tile[0] > 0 || cfg.mg_tile[1] > 0) {
    c->solver.mg_tile[0] = cfg.mg_tile[0] > 0 ? cfg.mg_tile[0] : 32;
    c->solver.mg_tile[1] = cfg.mg_tile[1] > 0 ? cfg.mg_tile[1] : 32;
  }
  c->solver.rb = c->rb;
  if ((rc = c->solver.setup(N, c->st))) { free_all(c); delete c; return rc; }
  c->solver.prof = &c->prof;
  c->solver.stream2 = c->st2;
  if (c->conc) {
    if (cudaStreamCreateWithFlags(&c->stm, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->evf, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->evj, cudaEventDisableTiming) != cudaSuccess) { free_all(c); delete c; return DROPLET_ERR_CUDA; }
    Solver& m = c->solver_m;
    m.f32_helm = c->solver.f32_helm;
    m.persistent = false;
    m.persist_pcg = true;
    m.spin_limit = c->solver.spin_limit;
    m.nsys_extra = na - 1;
    m.rb = c->rb;
    if ((rc = m.setup(N, c->stm))) { free_all(c); delete c; return rc; }
    m.prof = &c->prof;
    m.stream2 = c->st2;
    // SM budgets of the two branches' cooperative Jacobi-PCG launches: together at most the
    // SM count, so that both are co-resident; the momentum solve (the longer chain) gets 7/12
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    m.pcg_budget = std::max(1, nsm * 7 / 12);
    c->solver.pcg_budget = std::max(1, nsm - m.pcg_budget);
  }
  if (c->cfg.physics_mask & DROPLET_PHYS_FLOW) {
    int mm[3] = {g.n[0], g.n[1], g.n[2]};
    if ((rc = c->solver.prepare_mg(mm, c->cfg.precision == 1))) { free_all(c); delete c; return rc; }
  }
  cudaStream_t st = c->st;
  int gc = lin_grid(N);
  cudaMemsetAsync(c->scal, 0, sizeof(double) * SC_COUNT, st);
  cudaMemsetAsync(c->flags, 0, sizeof(unsigned), st);
  cudaMemsetAsync(c->dirty, 0, sizeof(int), st);
  cudaMemsetAsync(c->pr, 0, sizeof(double) * N, st);
  cudaMemsetAsync(c->mdot, 0, sizeof(double) * N, st);
  cudaMemsetAsync(c->mraw, 0, sizeof(double) * N, st);
  for (int a = 0; a < na; ++a) {
    cudaMemsetAsync(c->u[a], 0, sizeof(double) * nfaces(g, a), st);
    cudaMemsetAsync(c->us[a], 0, sizeof(double) * nfaces(g, a), st);
    cudaMemsetAsync(c->hu[a], 0, sizeof(double) * nfaces(g, a), st);
  }
  cudaMemsetAsync(c->hT, 0, sizeof(double) * N, st);
  cudaMemsetAsync(c->hW, 0, sizeof(double) * N, st);
  if (c->p.drl != 0.0) {
    if ((rc = dalloc(&c->expand, N))) { free_all(c); delete c; return rc; }
    cudaMemsetAsync(c->expand, 0, sizeof(double) * N, st);
  }
  reset_clock(c, st);
  if (cfg.co_max > 0.0) {
    c->p.dyn = c->scal;
    c->p.co_hmin = cfg.co_max * g.hmin;
  }
  ++g_launches, k_init<<<gc, TPB, 0, st>>>(g, c->p, c->alpha, c->T, c->omega, c->rhoG);
  ++g_launches, k_xi<<<gc, TPB, 0, st>>>(g, c->p, c->xi);
  if (g.bc[g.s][0] == BC_FORCED) {
    // inlet faces (index 0 along the streamwise axis) carry u_inflow: the first n0*n1 entries of u[s] in 3D,
    // the first n0 entries of u[1] in 2D
    long long cnt = g.axisym ? g.n[0] : (long long)g.n[0] * g.n[1];
    double* hv = (double*)malloc(sizeof(double) * cnt);
    for (long long q = 0; q < cnt; ++q) hv[q] = c->cfg.u_inflow;
    cudaMemcpyAsync(c->u[g.s], hv, sizeof(double) * cnt, cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
    free(hv);
  }
  if ((rc = run_diag(c, DIAG_INITIAL))) { free_all(c); delete c; return rc; }
  if (cudaStreamSynchronize(st) != cudaSuccess) { free_all(c); delete c; return DROPLET_ERR_CUDA; }
  *out = c;
  return 0;
}

static int one_step(dctx* c, int* nc_flag) {
  Geo& g = c->g;
  Phys& p = c->p;
  cudaStream_t st = c->st;
  long long N = g.N;
  int na = nact(g);
  int gc = lin_grid(N), nb = red_grid_cap(N, c->rb);
  double* u2 = c->u[2] ? c->u[2] : c->u[0];
  int mask = p.physics;
  // S0 (with the reset of the step's solver statistics)
  ++g_launches, k_thermo_pin<<<gc, TPB, 0, st>>>(g, p, c->alpha, c->T, c->omega, c->rhoG, c->rhoG_old, c->flags, c->dirty,
                                                 c->scal);
  if (c->s32.u[0]) {   // mixed precision: u^n in binary32 for the assembly stencils of this step
    const long long n0 = nfaces(g, 0), n1 = nfaces(g, 1), n2 = na == 3 ? nfaces(g, 2) : 0;
    ++g_launches, k_faces_f32<<<lin_grid(n0 + n1 + n2), TPB, 0, st>>>(c->u[0], c->u[1], na == 3 ? c->u[2] : c->u[0],
                                                                     c->s32.u[0], c->s32.u[1], c->s32.u[2], n0, n1, n2);
  }
  // S1, S2
  if (mask & DROPLET_PHYS_EVAP) {
    L_evap_raw(st, nb, g, p, c->alpha, c->omega, c->rhoG_old, c->T, c->u[0], c->u[1], u2, c->mraw, c->adj, c->part, c->flags);
    ++g_launches, k_evap_K<<<1, TPB, 0, st>>>(c->part, nb, c->scal, c->flags);
  } else {
    cudaMemsetAsync(c->mraw, 0, sizeof(double) * N, st);
    cudaMemsetAsync(c->scal + SC_K, 0, sizeof(double), st);
  }
  ++g_launches, k_alpha_source<<<gc, TPB, 0, st>>>(g, p, c->alpha, c->mraw, c->scal, c->T, c->expand, c->mdot, c->astar,
                                                   c->astar_f, c->flags, c->dirty);
  // S3, and S4 (the mixture properties) in the kernel that forms alpha^{n+1}
  const PropsOut po{c->rhoG_old, c->omega, c->T, c->rho, c->mu, c->kc, c->cp, c->Dm, c->s32, c->solid};
  if ((mask & DROPLET_PHYS_FLOW) && c->cfg.adv_scheme == 1) {
    // geometric advection, FP64 in both precisions: the planes in FL (normal) and AF[0]
    // (constant), the sweeps' intermediate alpha in aL and Rp
    double* const w[2] = {c->aL, c->Rp};
    double* const Nn[3] = {c->FL[0], c->FL[1], na == 3 ? c->FL[2] : nullptr};
    L_geo_advect(st, nb, g, p, c->astar, w, Nn, c->AF[0], c->u, c->alpha, c->part, po);
  } else if (mask & DROPLET_PHYS_FLOW) {
    if (c->cfg.precision == 1) {
      L_adv_faces_mx_all(st, g, p, c->astar, c->astar_f, c->u, c->FL, c->AF);
    } else {
      for (int a = 0; a < na; ++a)
        L_adv_faces(st, lin_grid(nfaces(g, a)), g, p, a, c->astar, c->u[a], c->FL[a], c->AF[a]);
    }
    double* F2 = c->FL[2] ? c->FL[2] : c->FL[0];
    double* A2 = c->AF[2] ? c->AF[2] : c->AF[0];
    ++g_launches, k_adv_low<<<gc, TPB, 0, st>>>(g, c->astar, c->FL[0], c->FL[1], F2, c->aL);
    L_adv_limit(st, gc, g, c->astar, c->aL, c->AF[0], c->AF[1], A2, c->Rp, c->Rm);
    L_adv_update(st, nb, g, p, c->aL, c->AF[0], c->AF[1], A2, c->Rp, c->Rm, c->alpha, c->part, c->flags, po);
  } else {
    ++g_launches, k_alpha_clip_only<<<nb, TPB, 0, st>>>(g, p, c->astar, c->alpha, c->part, po);
  }
  ++g_launches, k_clip_finish<<<1, TPB, 0, st>>>(c->part, nb, c->scal, c->flags);
  BoxSys bs;
  bs.D = c->bD; bs.b = c->brhs; bs.x = c->bx;
  for (int a = 0; a < 3; ++a) bs.c[a] = a < na ? c->bc[a] : nullptr;
  SolveStats ss;
  int rc;
  // S7 momentum predictor, on stream ms with solver sv: the components' box systems are
  // assembled from the old velocities (independent of S5 and S6), solved together in one
  // persistent launch where possible, and scattered into u*
  auto momentum = [&](cudaStream_t ms, Solver& sv) -> int {
    int nc7 = 0, rc7 = 0;
    SolveStats ss7;
    if (sv.persist_pcg && sv.nsys_extra == na - 1 && (c->conc || na == 1 || c->xb[na - 2][5])) {
      BoxSys sys[3];
      RecordSpec recs[3];
      for (int cc = 0; cc < na; ++cc) {
        int m[3] = {g.n[0], g.n[1], g.n[2]};
        m[cc] -= 1;
        long long nbx = (long long)m[0] * m[1] * m[2];
        BoxSys& b = sys[cc];
        if (cc == 0 && !c->conc) {
          b.D = c->bD; b.b = c->brhs; b.x = c->bx;
          for (int a = 0; a < 3; ++a) b.c[a] = a < na ? c->bc[a] : nullptr;
        } else {
          double* const* xs = c->xb[c->conc ? cc : cc - 1];
          b.D = xs[0]; b.b = xs[4]; b.x = xs[5];
          for (int a = 0; a < 3; ++a) b.c[a] = a < na ? xs[1 + a] : nullptr;
        }
        for (int a = 0; a < 3; ++a) b.m[a] = m[a];
        b.N = nbx;
        {
        ProfScope ps(&c->prof, KC_MOM_ASSEMBLE, ms, (12.0 + 2 * na) * nbx * 8.0);
        (c->cfg.precision == 1 ? L_mom_assemble_mx : L_mom_assemble)(
            ms, lin_grid(nbx), g, p, cc, c->u[0], c->u[1], u2, c->rho, c->mu, c->pr, c->alpha, c->xi, b.D, b.c[0],
            b.c[1], na == 3 ? b.c[2] : b.c[0], (double*)b.b, &c->s32);
        }
        L_faces_to_box(ms, lin_grid(nbx), g, cc, c->u[cc], b.x, c->hu[cc], c->scal);
        recs[cc] = RecordSpec{c->scal, SC_ITS_U, -1, cc > 0};
      }
      rc7 = sv.pcg_jacobi_multi(sys, na, c->cfg.helm_rtol, c->cfg.helm_maxit, recs, &ss7);
      if ((rc7 = soft_status(rc7, &nc7))) return rc7;
      for (int cc = 0; cc < na; ++cc) {
        cudaMemcpyAsync(c->us[cc], c->u[cc], sizeof(double) * nfaces(g, cc), cudaMemcpyDeviceToDevice, ms);
        L_mom_scatter(ms, lin_grid(nfaces(g, cc)), g, p, cc, sys[cc].x, c->us[cc]);
      }
      return nc7 == 2 ? DROPLET_ERR_TIMEOUT : nc7 ? DROPLET_ERR_NOT_CONVERGED : 0;
    }
    BoxSys bm = bs;
    bm.x = c->bx;
    for (int cc = 0; cc < na; ++cc) {
      int m[3] = {g.n[0], g.n[1], g.n[2]};
      m[cc] -= 1;
      long long nbx = (long long)m[0] * m[1] * m[2];
      {
      ProfScope ps(&c->prof, KC_MOM_ASSEMBLE, ms, (12.0 + 2 * na) * nbx * 8.0);
      (c->cfg.precision == 1 ? L_mom_assemble_mx : L_mom_assemble)(
          ms, lin_grid(nbx), g, p, cc, c->u[0], c->u[1], u2, c->rho, c->mu, c->pr, c->alpha, c->xi, c->bD, c->bc[0],
          c->bc[1], na == 3 ? c->bc[2] : c->bc[0], c->brhs, &c->s32);
      }
      for (int a = 0; a < 3; ++a) bm.m[a] = m[a];
      bm.N = nbx;
      L_faces_to_box(ms, lin_grid(nbx), g, cc, c->u[cc], c->bx, c->hu[cc], c->scal);
      sv.record_next(c->scal, SC_ITS_U, -1, cc > 0);
      rc7 = sv.pcg_jacobi(bm, c->cfg.helm_rtol, c->cfg.helm_maxit, &ss7);
      if ((rc7 = soft_status(rc7, &nc7))) return rc7;
      sv.record(c->scal, SC_ITS_U, -1, cc > 0);
      cudaMemcpyAsync(c->us[cc], c->u[cc], sizeof(double) * nfaces(g, cc), cudaMemcpyDeviceToDevice, ms);
      L_mom_scatter(ms, lin_grid(nfaces(g, cc)), g, p, cc, c->bx, c->us[cc]);
    }
    return nc7 == 2 ? DROPLET_ERR_TIMEOUT : nc7 ? DROPLET_ERR_NOT_CONVERGED : 0;
  };
  if (c->conc && (mask & DROPLET_PHYS_FLOW)) {   // fork: S7 on its own branch
    CKR(cudaEventRecord(c->evf, st));
    CKR(cudaStreamWaitEvent(c->stm, c->evf, 0));
    rc = momentum(c->stm, c->solver_m);
    if ((rc = soft_status(rc, nc_flag))) return rc;
    CKR(cudaEventRecord(c->evj, c->stm));
  }
  // S5 energy
  if ((mask & DROPLET_PHYS_ENERGY) && !p.const_props) {
    {
    ProfScope ps(&c->prof, KC_SCALAR_ASSEMBLE, st, (12.0 + 2 * na) * N * 8.0);
    (c->cfg.precision == 1 ? L_scalar_assemble_mx : L_scalar_assemble)(
        st, gc, g, p, 0, c->T, c->rho, c->cp, c->kc, c->Dm, c->mdot, c->u[0], c->u[1], u2, c->alpha, c->yq, p.T_amb,
        c->bD, c->bc[0], c->bc[1], na == 3 ? c->bc[2] : c->bc[0], c->brhs, &c->s32, c->omega);
    }
    for (int a = 0; a < 3; ++a) bs.m[a] = g.n[a];
    bs.N = N;
    bs.x = c->T;   // solved in place: T receives the solution
    ++g_launches, k_extrap<<<gc, TPB, 0, st>>>(N, c->T, c->hT, c->scal);
    c->solver.record_next(c->scal, SC_ITS_T, -1, 0);
    rc = c->solver.pcg_jacobi(bs, c->cfg.helm_rtol, c->cfg.helm_maxit, &ss);
    if ((rc = soft_status(rc, nc_flag))) return rc;
    c->solver.record(c->scal, SC_ITS_T, -1, 0);
    bs.x = c->bx;
  }
  // S6 species
  ++g_launches, k_yeq<<<gc, TPB, 0, st>>>(g, p, c->T, c->alpha, c->omega, c->yq, c->flags);
  if (mask & DROPLET_PHYS_SPECIES) {
    {
    ProfScope ps(&c->prof, KC_SCALAR_ASSEMBLE, st, (12.0 + 2 * na) * N * 8.0);
    (c->cfg.precision == 1 ? L_scalar_assemble_mx : L_scalar_assemble)(
        st, gc, g, p, 1, c->omega, c->rho, c->cp, c->kc, c->Dm, c->mdot, c->u[0], c->u[1], u2, c->alpha, c->yq, 0.0,
        c->bD, c->bc[0], c->bc[1], na == 3 ? c->bc[2] : c->bc[0], c->brhs, &c->s32, nullptr);
    }
    for (int a = 0; a < 3; ++a) bs.m[a] = g.n[a];
    bs.N = N;
    bs.x = c->omega;   // in place
    ++g_launches, k_extrap<<<gc, TPB, 0, st>>>(N, c->omega, c->hW, c->scal);
    c->solver.record_next(c->scal, SC_ITS_W, -1, 0);
    rc = c->solver.pcg_jacobi(bs, c->cfg.helm_rtol, c->cfg.helm_maxit, &ss);
    if ((rc = soft_status(rc, nc_flag))) return rc;
    c->solver.record(c->scal, SC_ITS_W, -1, 0);
    bs.x = c->bx;
  } else {
    ++g_launches, k_species_noflow<<<gc, TPB, 0, st>>>(g, c->alpha, c->yq, c->omega);
  }
  ++g_launches, k_rhoG<<<gc, TPB, 0, st>>>(g, p, c->T, c->omega, c->rhoG);
  // S7 - S10
  if (mask & DROPLET_PHYS_FLOW) {
    if (c->conc) {
      CKR(cudaStreamWaitEvent(st, c->evj, 0));   // join the momentum branch
    } else {
      rc = momentum(st, c->solver);
      if ((rc = soft_status(rc, nc_flag))) return rc;
    }
    double* us2 = c->us[2] ? c->us[2] : c->us[0];
    // T^n: the history field the energy solve's guess kept, or T itself when T is not solved
    const double* T0 = ((mask & DROPLET_PHYS_ENERGY) && !p.const_props) ? c->hT : c->T;
    L_poisson_assemble(st, gc, g, p, c->mdot, c->alpha, c->rhoG_old, c->rhoG, c->u[0], c->u[1], u2,
                                           c->us[0], c->us[1], us2, c->rho, c->T, T0, c->expand, c->S, c->bD, c->bc[0], c->bc[1],
                                           na == 3 ? c->bc[2] : c->bc[0], c->brhs, c->dp);
    for (int a = 0; a < 3; ++a) bs.m[a] = g.n[a];
    bs.N = N;
    bs.x = c->dp;   // pressure increment from a zero initial guess (set by the assembly), solved in place
    c->solver.record_next(c->scal, SC_ITS_P, SC_RES_P, 0);
    rc = c->solver.pcg_mg(bs, c->cfg.cg_rtol, c->cfg.cg_maxit, c->cfg.precision == 1, &ss);
    if ((rc = soft_status(rc, nc_flag))) return rc;
    c->solver.record(c->scal, SC_ITS_P, SC_RES_P, 0);
    bs.x = c->bx;
    L_correct_all(st, g, p, c->us, c->dp, c->rho, c->u, c->pr);
  } else {
    cudaMemsetAsync(c->dp, 0, sizeof(double) * N, st);
    cudaMemsetAsync(c->S, 0, sizeof(double) * N, st);
  }
  // S11
  if ((rc = run_diag(c, DIAG_STEP_END))) return rc;
  CKR(cudaGetLastError());
  return 0;
}

// ---------------------------------------------------------------- the public context
struct droplet_ctx {
  cudaStream_t st = nullptr;         // the caller's stream (or own_main)
  cudaStream_t own_main = nullptr;   // internal stream when the caller passed the legacy default stream
  std::vector<dctx*> d;              // one context per droplet
  std::vector<cudaEvent_t> ev;       // fork / join events of the batch graph
  cudaGraphExec_t exec = nullptr;    // the captured step of every droplet
  double* hnc = nullptr;             // pinned not-converged marks
  bool prof_on = false;
  int rb = RED_BLOCKS;               // reduction block cap in use
};

static void free_ctx(droplet_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  for (auto x : c->d) {
    if (x->st) cudaStreamSynchronize(x->st);
    free_all(x);
    delete x;
  }
  c->d.clear();
  for (auto e : c->ev) cudaEventDestroy(e);
  c->ev.clear();
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->hnc) cudaFreeHost(c->hnc);
  if (c->own_main) cudaStreamDestroy(c->own_main);
  delete c;
}

// Capture one step of every droplet into one graph: each droplet is a branch forked from
// the main stream (every stage, every solver loop as a conditional WHILE node) and joined back.
static int capture_step(droplet_ctx* c) {
  cudaGraph_t graph = nullptr;
  int nc = 0, rc = 0;
  bool batch = c->d.size() > 1;
  CKR(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeRelaxed));
  if (batch) CKR(cudaEventRecord(c->ev[0], c->st));
  for (size_t i = 0; i < c->d.size() && !rc; ++i) {
    dctx* x = c->d[i];
    if (batch) cudaStreamWaitEvent(x->st, c->ev[0], 0);
    x->solver.capturing = x->solver_m.capturing = true;
    rc = one_step(x, &nc);
    x->solver.capturing = x->solver_m.capturing = false;
    if (batch) {
      cudaEventRecord(c->ev[1 + i], x->st);
      cudaStreamWaitEvent(c->st, c->ev[1 + i], 0);
    }
  }
  cudaError_t e = cudaStreamEndCapture(c->st, &graph);
  if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
  CKR(e);
  e = cudaGraphInstantiate(&c->exec, graph, 0);
  cudaGraphDestroy(graph);
  CKR(e);
  return 0;
}

static void set_rb(droplet_ctx* c, int rb) {
  c->rb = rb;
  for (auto x : c->d) { x->rb = rb; x->solver.rb = rb; }
}

// Autotuner.  (1) The tile shape of the persistent multigrid's temporal blocking (2D
// hierarchies): larger tiles cut the halo overhead and the number of tiles a block runs
// in turn, smaller ones spread a level over more blocks.  (2) For batches, the block cap
// of the launched reduction kernels, so that the branches of the batch graph share the
// SMs.  Each candidate is captured and timed over a few steps on copies of the state;
// the fastest is kept and the state restored.
static int autotune(droplet_ctx* c) {
  // snapshot the state of every droplet
  std::vector<std::vector<double*>> snap(c->d.size());
  auto fields = [](dctx* x, double* fs[8]) {
    double* f[8] = {x->alpha, x->T, x->omega, x->pr, x->rhoG, x->u[0], x->u[1], x->u[2]};
    for (int q = 0; q < 8; ++q) fs[q] = f[q];
  };
  for (size_t i = 0; i < c->d.size(); ++i) {
    dctx* x = c->d[i];
    double* fs[8];
    fields(x, fs);
    for (int f = 0; f < 8; ++f) {
      if (!fs[f]) { snap[i].push_back(nullptr); continue; }
      long long n = f < 5 ? x->g.N : nfaces(x->g, f - 5);
      double* q = nullptr;
      if (cudaMalloc(&q, sizeof(double) * n) != cudaSuccess) return DROPLET_ERR_NOMEM;
      cudaMemcpyAsync(q, fs[f], sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st);
      snap[i].push_back(q);
    }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = 0;
  // time three graph steps of the current settings, then put the state back
  auto trial = [&](float* ms) -> int {
    if (c->exec) { cudaGraphExecDestroy(c->exec); c->exec = nullptr; }
    int r = capture_step(c);
    if (r) return r;
    CKR(cudaGraphLaunch(c->exec, c->st));   // warm-up
    CKR(cudaEventRecord(e0, c->st));
    for (int k = 0; k < 3; ++k) CKR(cudaGraphLaunch(c->exec, c->st));
    CKR(cudaEventRecord(e1, c->st));
    CKR(cudaEventSynchronize(e1));
    cudaEventElapsedTime(ms, e0, e1);
    for (size_t i = 0; i < c->d.size(); ++i) {
      dctx* x = c->d[i];
      double* fs[8];
      fields(x, fs);
      for (int f = 0; f < 8; ++f) {
        if (!fs[f]) continue;
        long long n = f < 5 ? x->g.N : nfaces(x->g, f - 5);
        cudaMemcpyAsync(fs[f], snap[i][f], sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st);
      }
      cudaMemsetAsync(x->scal, 0, sizeof(double) * SC_COUNT, c->st);
      reset_clock(x, c->st);
      cudaMemsetAsync(x->flags, 0, sizeof(unsigned), c->st);
      cudaMemsetAsync(x->dirty, 0xff, sizeof(int), c->st);
    }
    CKR(cudaStreamSynchronize(c->st));
    return 0;
  };
  bool tiles = false;
  auto fixed_tile = [](const dctx* x) { return x->cfg.mg_tile[0] > 0 || x->cfg.mg_tile[1] > 0; };
  for (auto x : c->d)
    tiles = tiles || (x->solver.persistent && (x->cfg.physics_mask & DROPLET_PHYS_FLOW) && x->g.n[2] == 1 &&
                      !fixed_tile(x));
  if (tiles) {
    const int cand[][2] = {{32, 32}, {64, 32}, {64, 64}, {128, 32}};
    float best = 1e30f;
    int bt = 0;
    for (int k = 0; k < 4 && !rc; ++k) {
      for (auto x : c->d)
        if (!fixed_tile(x)) { x->solver.mg_tile[0] = cand[k][0]; x->solver.mg_tile[1] = cand[k][1]; }
      float ms = 0.f;
      rc = trial(&ms);
      if (!rc && ms < best) { best = ms; bt = k; }
    }
    for (auto x : c->d)
      if (!fixed_tile(x)) { x->solver.mg_tile[0] = cand[bt][0]; x->solver.mg_tile[1] = cand[bt][1]; }
  }
  if (c->d.size() > 1 && !rc) {
    const int cand[] = {RED_BLOCKS, 304, 152, 76, 38};
    float best = 1e30f;
    int best_rb = RED_BLOCKS;
    for (int rb : cand) {
      set_rb(c, rb);
      float ms = 0.f;
      rc = trial(&ms);
      if (rc) break;
      if (ms < best) { best = ms; best_rb = rb; }
    }
    set_rb(c, best_rb);
  }
  for (auto& v : snap) for (auto q : v) cudaFree(q);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (c->exec) { cudaGraphExecDestroy(c->exec); c->exec = nullptr; }
  for (auto x : c->d) if (run_diag(x, DIAG_INITIAL)) return DROPLET_ERR_CUDA;
  CKR(cudaStreamSynchronize(c->st));
  return 0;
}

extern "C" int droplet_init(const droplet_config* cfgs, int n_droplets, void* cuda_stream, droplet_ctx** out) {
  if (!cfgs || !out || n_droplets < 1 || n_droplets > 4096) return DROPLET_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n_droplets; ++i) {
    int rc = check_cfg(cfgs[i]);
    if (rc) return rc;
  }
  droplet_ctx* c = new (std::nothrow) droplet_ctx();
  if (!c) return DROPLET_ERR_NOMEM;
  c->st = (cudaStream_t)cuda_stream;
  if (!c->st) {
    // the legacy default stream cannot be captured: work on an internal blocking stream,
    // which the legacy default stream orders against all other work
    if (cudaStreamCreate(&c->own_main) != cudaSuccess) { delete c; return DROPLET_ERR_CUDA; }
    c->st = c->own_main;
  }
  if (cudaMallocHost((void**)&c->hnc, sizeof(double) * n_droplets) != cudaSuccess) { free_ctx(c); return DROPLET_ERR_NOMEM; }
  bool batch = n_droplets > 1;
  for (int i = 0; i < n_droplets; ++i) {
    dctx* x = nullptr;
    int rc = init_one(cfgs[i], c->st, batch, &x);
    if (rc) { free_ctx(c); return rc; }
    c->d.push_back(x);
  }
  if (batch) {
    // SM budgets of the persistent solvers: proportional to the cells, at least one SM
    // each, summing to at most the SM count, so that the cooperative solves of all
    // droplets, running concurrently on the branches of the step graph, are co-resident
    // at once; with more droplets than SMs the batch uses the launched solvers.
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    bool persist = n_droplets <= nsm;
    for (auto x : c->d) persist = persist && x->solver.persistent;
    if (persist) {
      double tot = 0.0;
      for (auto x : c->d) tot += (double)x->g.N;
      std::vector<int> bud(n_droplets);
      int sum = 0;
      for (int i = 0; i < n_droplets; ++i) {
        bud[i] = std::max(1, (int)std::floor(nsm * (double)c->d[i]->g.N / tot));
        sum += bud[i];
      }
      while (sum > nsm) {   // trim the largest budgets
        int k = (int)(std::max_element(bud.begin(), bud.end()) - bud.begin());
        --bud[k];
        --sum;
      }
      for (int i = 0; i < n_droplets; ++i) c->d[i]->solver.sm_budget = bud[i];
    } else {
      for (auto x : c->d) x->solver.persistent = x->solver.persist_pcg = false;
    }
    c->ev.resize(n_droplets + 1);
    for (auto& e : c->ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) { free_ctx(c); return DROPLET_ERR_CUDA; }
  }
  // batches, and single 2D droplets with flow large enough for the tile shape to matter
  const dctx* x0 = c->d[0];
  if (batch || (x0->solver.persistent && (x0->cfg.physics_mask & DROPLET_PHYS_FLOW) && x0->g.n[2] == 1 &&
                x0->g.N >= 32768 && x0->cfg.mg_tile[0] == 0 && x0->cfg.mg_tile[1] == 0)) {
    int rc = autotune(c);
    if (rc) { free_ctx(c); return rc; }
  }
  *out = c;
  return 0;
}

extern "C" int droplet_step(droplet_ctx* c, int n_steps) {
  if (!c || n_steps < 0) return DROPLET_ERR_ARG;
  int nc = 0;
  for (auto x : c->d) CKR(cudaMemsetAsync(x->scal + SC_NC, 0, sizeof(double), x->st));
  for (auto x : c->d) if (x->st != c->st) CKR(cudaStreamSynchronize(x->st));
  if (c->prof_on) {
    // timed kernel classes need one event pair per launch: run the stages directly
    for (int s = 0; s < n_steps; ++s)
      for (auto x : c->d) {
        int rc = one_step(x, &nc);
        if (rc) return rc;
        x->step += 1;
      }
    for (auto x : c->d) if (x->st != c->st) CKR(cudaStreamSynchronize(x->st));
  } else {
    if (!c->exec) {
      int rc = capture_step(c);
      if (rc) return rc;
    }
    for (int s = 0; s < n_steps; ++s) {
      CKR(cudaGraphLaunch(c->exec, c->st));
      for (auto x : c->d) x->step += 1;
    }
  }
  for (size_t i = 0; i < c->d.size(); ++i)
    CKR(cudaMemcpyAsync(c->hnc + i, c->d[i]->scal + SC_NC, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CKR(cudaStreamSynchronize(c->st));
  for (size_t i = 0; i < c->d.size(); ++i) {
    if (c->hnc[i] >= 2.0) nc = 2;
    else if (c->hnc[i] != 0.0 && nc < 1) nc = 1;
  }
  return nc == 2 ? DROPLET_ERR_TIMEOUT : nc ? DROPLET_ERR_NOT_CONVERGED : 0;
}

extern "C" int droplet_profile(droplet_ctx* c, int enable) {
  if (!c) return DROPLET_ERR_ARG;
  CKR(cudaStreamSynchronize(c->st));
  for (auto x : c->d) {
    CKR(cudaStreamSynchronize(x->st));
    if (enable) x->prof.reset();
    x->prof.on = enable != 0;
  }
  c->prof_on = enable != 0;
  return 0;
}

extern "C" int droplet_profile_read(droplet_ctx* c, int kclass, double* ms, long long* launches, double* bytes,
                                    double* flops64) {
  if (!c || !ms || !launches || !bytes || kclass < 0 || kclass >= KC_COUNT) return DROPLET_ERR_ARG;
  double tm = 0.0, tb = 0.0, tf = 0.0;
  long long tn = 0;
  for (auto x : c->d) {
    double m, b, f;
    long long n;
    int rc = x->prof.read(kclass, &m, &n, &b, &f);
    if (rc) return rc;
    tm += m; tb += b; tn += n; tf += f;
  }
  *ms = tm; *launches = tn; *bytes = tb;
  if (flops64) *flops64 = tf;
  return 0;
}

extern "C" int droplet_launch_count(droplet_ctx* c, long long* launches) {
  if (!c || !launches) return DROPLET_ERR_ARG;
  *launches = g_launches;
  return 0;
}

extern "C" int droplet_sync(droplet_ctx* c) {
  if (!c) return DROPLET_ERR_ARG;
  CKR(cudaStreamSynchronize(c->st));
  for (auto x : c->d) CKR(cudaStreamSynchronize(x->st));
  return 0;
}

extern "C" int droplet_diag(droplet_ctx* cc, int droplet, droplet_diag_t* out) {
  if (!cc || !out || droplet < 0 || droplet >= (int)cc->d.size()) return DROPLET_ERR_ARG;
  dctx* c = cc->d[droplet];
  CKR(cudaStreamSynchronize(cc->st));
  CKR(cudaMemcpyAsync(c->hscal, c->scal, sizeof(double) * SC_COUNT, cudaMemcpyDeviceToHost, c->st));
  CKR(cudaMemcpyAsync(c->hflags, c->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, c->st));
  CKR(cudaMemsetAsync(c->flags, 0, sizeof(unsigned), c->st));
  CKR(cudaStreamSynchronize(c->st));
  const double* s = c->hscal;
  double w = c->g.axisym ? 2.0 * M_PI : 1.0;
  memset(out, 0, sizeof(*out));
  out->t = s[SC_TIME];
  out->step = c->step;
  out->V_l = w * s[SC_SUM_ALPHA_V];
  out->d_eq = cbrt(6.0 * out->V_l / M_PI);
  out->d2 = out->d_eq * out->d_eq;
  out->mdot_tot = w * s[SC_SUM_MDOT_V];
  out->K_norm = s[SC_K];
  out->T_s_mean = s[SC_SUM_G] > 0.0 ? s[SC_SUM_TG] / s[SC_SUM_G] : 0.0;
  out->M_liq = c->p.drl == 0.0 ? c->cfg.rho_l * out->V_l : w * s[SC_SUM_MLIQ];
  out->M_vap = w * s[SC_SUM_VAP];
  out->vap_out_cum = w * s[SC_VAPOUT];
  out->max_u = s[SC_MAXU];
  out->alpha_min = s[SC_AMIN];
  out->alpha_max = s[SC_AMAX];
  out->clip_mass = w * s[SC_CLIP];
  out->its_p = (int)s[SC_ITS_P]; out->its_T = (int)s[SC_ITS_T]; out->its_w = (int)s[SC_ITS_W];
  out->its_u = (int)s[SC_ITS_U];
  out->res_p = s[SC_RES_P];
  out->flags = *c->hflags;
  if (out->flags & DROPLET_FLAG_NONFINITE) return DROPLET_ERR_NONFINITE;
  const double chk[] = {out->V_l, out->mdot_tot, out->K_norm, out->T_s_mean, out->M_vap, out->vap_out_cum,
                        out->max_u, out->alpha_min, out->alpha_max, out->clip_mass, out->res_p};
  for (double v : chk)
    if (!std::isfinite(v)) return DROPLET_ERR_NONFINITE;
  return 0;
}

static double* field_ptr(dctx* c, int id, long long* n, bool* writable) {
  Geo& g = c->g;
  *writable = false;
  *n = g.N;
  switch (id) {
    case DROPLET_F_ALPHA: *writable = true; return c->alpha;
    case DROPLET_F_T: *writable = true; return c->T;
    case DROPLET_F_OMEGA: *writable = true; return c->omega;
    case DROPLET_F_P: *writable = true; return c->pr;
    case DROPLET_F_RHOG: *writable = true; return c->rhoG;
    case DROPLET_F_MDOT: return c->mdot;
    case DROPLET_F_MRAW: return c->mraw;
    case DROPLET_F_ALPHA_STAR: return c->astar;
    case DROPLET_F_DP: return c->dp;
    case DROPLET_F_S: return c->S;
    case DROPLET_F_RHOG_OLD: return c->rhoG_old;
    case DROPLET_F_OMEGA_PINNED: return nullptr;
    case DROPLET_F_EXPAND: *writable = true; return c->expand;   // (null: constant liquid density)
    default: break;
  }
  int a = -1;
  bool star = false;
  if (id >= DROPLET_F_U0 && id <= DROPLET_F_U2) a = id - DROPLET_F_U0;
  if (id >= DROPLET_F_USTAR0 && id <= DROPLET_F_USTAR2) { a = id - DROPLET_F_USTAR0; star = true; }
  if (a < 0 || a >= nact(g)) return nullptr;
  *n = nfaces(g, a);
  *writable = !star;
  return star ? c->us[a] : c->u[a];
}

extern "C" int droplet_field_size(droplet_ctx* cc, int droplet, int field_id, size_t* n) {
  if (!cc || !n || droplet < 0 || droplet >= (int)cc->d.size()) return DROPLET_ERR_ARG;
  long long m;
  bool w;
  if (!field_ptr(cc->d[droplet], field_id, &m, &w)) return DROPLET_ERR_ARG;
  *n = (size_t)m;
  return 0;
}

extern "C" int droplet_get_field(droplet_ctx* cc, int droplet, int field_id, double* host, size_t n) {
  if (!cc || !host || droplet < 0 || droplet >= (int)cc->d.size()) return DROPLET_ERR_ARG;
  dctx* c = cc->d[droplet];
  long long m;
  bool w;
  double* d = field_ptr(c, field_id, &m, &w);
  if (!d) return DROPLET_ERR_ARG;
  if ((size_t)m != n) return DROPLET_ERR_SIZE;
  CKR(cudaStreamSynchronize(cc->st));
  CKR(cudaMemcpyAsync(host, d, sizeof(double) * n, cudaMemcpyDeviceToHost, c->st));
  CKR(cudaStreamSynchronize(c->st));
  return 0;
}

extern "C" int droplet_set_field(droplet_ctx* cc, int droplet, int field_id, const double* host, size_t n) {
  if (!cc || !host || droplet < 0 || droplet >= (int)cc->d.size()) return DROPLET_ERR_ARG;
  dctx* c = cc->d[droplet];
  long long m;
  bool w;
  double* d = field_ptr(c, field_id, &m, &w);
  if (!d || !w) return DROPLET_ERR_ARG;
  if ((size_t)m != n) return DROPLET_ERR_SIZE;
  CKR(cudaStreamSynchronize(cc->st));
  CKR(cudaMemcpyAsync(d, host, sizeof(double) * n, cudaMemcpyHostToDevice, c->st));
  CKR(cudaMemsetAsync(c->dirty, 0xff, sizeof(int), c->st));
  CKR(cudaMemsetAsync(c->scal + SC_HIST, 0, sizeof(double), c->st));   // no previous step for this state
  CKR(cudaStreamSynchronize(c->st));
  return 0;
}

extern "C" void droplet_free(droplet_ctx* c) { free_ctx(c); }

// ---------------------------------------------------------------- adjoint (no flow)
static int adjoint_flow(droplet_ctx* cc, int n_steps, int ckpt_every, double* J, double* dJ_dTamb, double* dJ_dDg,
                        double* dJ_dT0, size_t nT0);
extern "C" int droplet_adjoint(droplet_ctx* cc, int n_steps, int ckpt_every, double* J, double* dJ_dTamb,
                               double* dJ_dDg, double* dJ_dT0, size_t nT0) {
  if (!cc || cc->d.size() != 1 || n_steps < 1 || ckpt_every < 1 || !J) return DROPLET_ERR_ARG;
  dctx* x = cc->d[0];
  const droplet_config& cf = x->cfg;
  if (cf.physics_mask & DROPLET_PHYS_FLOW) return adjoint_flow(cc, n_steps, ckpt_every, J, dJ_dTamb, dJ_dDg, dJ_dT0, nT0);
  if (cf.physics_mask != (DROPLET_PHYS_EVAP | DROPLET_PHYS_ENERGY | DROPLET_PHYS_SPECIES) || cf.precision != 0 ||
      cf.eq_model != 0 || cf.const_props_check != 0 || cf.bc_mode != 0 || cf.co_max != 0.0 || cf.drho_l_dT != 0.0 ||
      cf.fiber != 0 || cf.cp_v != cf.cp_g || x->step != 0)
    return DROPLET_ERR_ARG;
  Geo& g = x->g;
  Phys& p = x->p;
  long long N = g.N;
  if (dJ_dT0 && nT0 != (size_t)N) return DROPLET_ERR_SIZE;
  cudaStream_t st = x->st;
  CKR(cudaStreamSynchronize(cc->st));
  CKR(cudaStreamSynchronize(st));
  int nseg = (n_steps + ckpt_every - 1) / ckpt_every;
  size_t S3 = 3 * (size_t)N;
  // device work memory
  double *ck = nullptr, *seg = nullptr, *w = nullptr, *acc = nullptr, *part = nullptr, *fin = nullptr;
  const int NW = 17;
  auto cleanup = [&]() { cudaFree(ck); cudaFree(seg); cudaFree(w); cudaFree(acc); cudaFree(part); cudaFree(fin); };
  if (cudaMalloc(&ck, sizeof(double) * S3 * nseg) != cudaSuccess || cudaMalloc(&seg, sizeof(double) * S3 * (ckpt_every + 1)) != cudaSuccess ||
      cudaMalloc(&w, sizeof(double) * N * NW) != cudaSuccess || cudaMalloc(&acc, sizeof(double) * AC_COUNT) != cudaSuccess ||
      cudaMalloc(&part, sizeof(double) * RED_BLOCKS * 4) != cudaSuccess || cudaMalloc(&fin, sizeof(double) * S3) != cudaSuccess) {
    cleanup();
    return DROPLET_ERR_NOMEM;
  }
  double* aA = w;           double* aT = w + N;       double* aW = w + 2 * N;
  double* Tn1bar = w + 3 * N; double* wpbar = w + 4 * N; double* rhobar = w + 5 * N;
  double* Dbar = w + 6 * N;  double* kbar = w + 7 * N;  double* cpbar = w + 8 * N;
  double* mdbar = w + 9 * N; double* rgbar = w + 10 * N; double* mrbar = w + 11 * N;
  double* aAn = w + 12 * N;  double* Tnbar = w + 13 * N; double* wp = w + 14 * N;
  double* zero = w + 15 * N;
  cudaMemsetAsync(acc, 0, sizeof(double) * AC_COUNT, st);
  cudaMemsetAsync(zero, 0, sizeof(double) * N, st);
  double wgt = g.axisym ? 2.0 * M_PI : 1.0;
  double jweight = wgt / n_steps;
  auto save_state = [&](double* dst) {
    cudaMemcpyAsync(dst, x->alpha, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(dst + N, x->T, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(dst + 2 * N, x->omega, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  };
  auto load_state = [&](const double* src) {
    cudaMemcpyAsync(x->alpha, src, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(x->T, src + N, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(x->omega, src + 2 * N, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(x->dirty, 0xff, sizeof(int), st);   // rho_G from T and omega at S0
  };
  // every forward step starts from its state alone (no extrapolated guesses), so that
  // the steps recomputed from the checkpoints repeat the first pass bit for bit
  auto step_alone = [&](int* ncp) {
    cudaMemsetAsync(x->scal + SC_HIST, 0, sizeof(double), st);
    return one_step(x, ncp);
  };
  int nc = 0, rc = 0;
  // forward with checkpoints every ckpt_every steps, J accumulated on the device
  for (int n = 0; n < n_steps && !rc; ++n) {
    if (n % ckpt_every == 0) save_state(ck + S3 * (n / ckpt_every));
    rc = step_alone(&nc);
    L_acc_J(st, x->scal, jweight, acc);
  }
  save_state(fin);
  CKR(cudaStreamSynchronize(st));
  double host_acc[AC_COUNT];
  CKR(cudaMemcpy(host_acc, acc, sizeof(double) * AC_COUNT, cudaMemcpyDeviceToHost));
  *J = host_acc[AC_J];
  bool want = dJ_dTamb || dJ_dDg || dJ_dT0;
  if (!rc && want) {
    cudaMemsetAsync(aA, 0, sizeof(double) * 3 * N, st);   // aA, aT, aW: J does not depend on the final state
    BoxSys bs;
    bs.D = x->bD; bs.b = x->brhs; bs.x = x->bx;
    int na = nact(g);
    for (int a = 0; a < 3; ++a) { bs.c[a] = a < na ? x->bc[a] : nullptr; bs.m[a] = g.n[a]; }
    bs.N = N;
    double* u2 = x->u[2] ? x->u[2] : x->u[0];
    SolveStats ss;
    for (int sgi = nseg - 1; sgi >= 0 && !rc; --sgi) {
      int n0 = sgi * ckpt_every, n1 = n0 + ckpt_every < n_steps ? n0 + ckpt_every : n_steps;
      // states n0 .. n1-1 of the segment
      load_state(ck + S3 * sgi);
      for (int n = n0; n < n1 && !rc; ++n) {
        save_state(seg + S3 * (n - n0));
        if (n + 1 < n1) rc = step_alone(&nc);
      }
      for (int n = n1 - 1; n >= n0 && !rc; --n) {
        const double* sA = seg + S3 * (n - n0);
        const double* sT = sA + N;
        const double* sW = sA + 2 * N;
        load_state(sA);
        rc = step_alone(&nc);            // leaves step n's intermediates and state n+1
        if (rc) break;
        L_adj_pin(st, g, p, sA, sT, sW, wp);
        // species: adjoint solve on the free rows, pinned rows and coefficients
        L_scalar_assemble(st, lin_grid(N), g, p, 1, wp, x->rho, x->cp, x->kc, x->Dm, x->mdot, x->u[0], x->u[1], u2,
                          x->alpha, x->yq, 0.0, x->bD, x->bc[0], x->bc[1], na == 3 ? x->bc[2] : x->bc[0], x->brhs,
                          nullptr);
        L_adj_rhs(st, g, aW, x->alpha, 1, x->brhs, x->bx);
        rc = x->solver.pcg_jacobi(bs, 1e-14, 4 * cf.helm_maxit, &ss);
        if (rc == DROPLET_ERR_NOT_CONVERGED) { nc = 1; rc = 0; }
        if (rc) break;
        L_adj_species(st, g, p, x->bx, aW, aT, x->alpha, wp, x->omega, x->T, x->rho, x->Dm, Tn1bar, wpbar, rhobar, Dbar);
        // energy
        L_scalar_assemble(st, lin_grid(N), g, p, 0, sT, x->rho, x->cp, x->kc, x->Dm, x->mdot, x->u[0], x->u[1], u2,
                          x->alpha, x->yq, p.T_amb, x->bD, x->bc[0], x->bc[1], na == 3 ? x->bc[2] : x->bc[0], x->brhs,
                          nullptr);
        L_adj_rhs(st, g, Tn1bar, x->alpha, 0, x->brhs, x->bx);
        rc = x->solver.pcg_jacobi(bs, 1e-14, 4 * cf.helm_maxit, &ss);
        if (rc == DROPLET_ERR_NOT_CONVERGED) { nc = 1; rc = 0; }
        if (rc) break;
        L_adj_energy(st, g, p, x->bx, sT, x->T, x->rho, x->cp, x->kc, Tnbar, rhobar, kbar, cpbar, mdbar);
        // properties, clipping, alpha source, J, cap, K and f(alpha)
        L_adj_source(st, g, p, aA, sA, x->alpha, x->astar, x->rhoG_old, x->mraw, x->scal, rhobar, kbar, cpbar, Dbar,
                     jweight, aAn, rgbar, mdbar, mrbar, part, acc);
        // evaporation flux at the adjacent gas cells
        L_adj_evap(st, g, p, sA, wp, x->rhoG_old, x->adj, mrbar, aAn, wpbar, rgbar, part, acc);
        // gas density and the pinned liquid values of S0
        L_adj_thermo(st, g, p, sA, sT, wp, x->rhoG_old, rgbar, wpbar, Tnbar, aW);
        cudaMemcpyAsync(aA, aAn, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(aT, Tnbar, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
        CKR(cudaGetLastError());
      }
    }
    if (!rc) {
      L_adj_tamb(st, g, p, aT, part, acc);
      CKR(cudaStreamSynchronize(st));
      CKR(cudaMemcpy(host_acc, acc, sizeof(double) * AC_COUNT, cudaMemcpyDeviceToHost));
      if (dJ_dDg) *dJ_dDg = host_acc[AC_DGAS] * (1.0e5 / cf.P);
      if (dJ_dTamb) *dJ_dTamb = host_acc[AC_TAMB];
      if (dJ_dT0) CKR(cudaMemcpy(dJ_dT0, aT, sizeof(double) * N, cudaMemcpyDeviceToHost));
    }
  }
  // leave the context at the state after n_steps
  load_state(fin);
  CKR(cudaStreamSynchronize(st));
  cleanup();
  {
    const double tn = n_steps * p.dt;   // the clock the forward and recomputed steps advanced
    CKR(cudaMemcpy(x->scal + SC_TIME, &tn, sizeof(double), cudaMemcpyHostToDevice));
  }
  x->step = n_steps;
  if (rc) return rc;
  return nc ? DROPLET_ERR_NOT_CONVERGED : 0;
}

// ---------------------------------------------------------------- adjoint with flow
// The state of a step as the flow adjoint keeps it: alpha, T, omega, p_rgh (cells), then the
// face velocities of each active direction.
static long long flow_state_size(const dctx* x) {
  long long s = 4 * x->g.N;
  for (int a = 0; a < nact(x->g); ++a) s += nfaces(x->g, a);
  return s;
}
static void flow_save(dctx* x, double* dst) {
  const long long N = x->g.N;
  cudaStream_t st = x->st;
  cudaMemcpyAsync(dst, x->alpha, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(dst + N, x->T, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(dst + 2 * N, x->omega, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(dst + 3 * N, x->pr, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  long long o = 4 * N;
  for (int a = 0; a < nact(x->g); ++a) {
    cudaMemcpyAsync(dst + o, x->u[a], sizeof(double) * nfaces(x->g, a), cudaMemcpyDeviceToDevice, st);
    o += nfaces(x->g, a);
  }
}
// load a state; S0 then re-evaluates rho_G from it and the solves start from it alone, so
// that a recomputed step repeats the first pass bit for bit
static void flow_load(dctx* x, const double* src) {
  const long long N = x->g.N;
  cudaStream_t st = x->st;
  cudaMemcpyAsync(x->alpha, src, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(x->T, src + N, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(x->omega, src + 2 * N, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(x->pr, src + 3 * N, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  long long o = 4 * N;
  for (int a = 0; a < nact(x->g); ++a) {
    cudaMemcpyAsync(x->u[a], src + o, sizeof(double) * nfaces(x->g, a), cudaMemcpyDeviceToDevice, st);
    o += nfaces(x->g, a);
  }
  cudaMemsetAsync(x->dirty, 0xff, sizeof(int), st);
}
static int flow_step_alone(dctx* x, int* nc) {
  cudaMemsetAsync(x->scal + SC_HIST, 0, sizeof(double), x->st);
  return one_step(x, nc);
}

// Work memory of the flow adjoint: the adjoints of every stage input (AdjArr order), of the
// state before and after the step, and the scratch of the adjoint solves
struct FlowWork {
  double* lam[J_COUNT] = {};
  double *lA = nullptr, *lT = nullptr, *lW = nullptr, *lP = nullptr, *lU[3] = {nullptr, nullptr, nullptr};
  double *lT1 = nullptr, *lW1 = nullptr;     // adjoints of T^{n+1}, omega^{n+1} within the step
  const double *sA = nullptr, *sT = nullptr, *sW = nullptr, *sP = nullptr, *sU[3] = {nullptr, nullptr, nullptr};
  double *wp = nullptr, *mu = nullptr, *bxa = nullptr, *bmu = nullptr, *mrbar = nullptr, *scr1 = nullptr,
         *scr2 = nullptr, *part = nullptr, *acc = nullptr;
  std::vector<double*> owned;
  int get(double** q, long long n) {
    if (cudaMalloc((void**)q, sizeof(double) * (size_t)(n > 0 ? n : 1)) != cudaSuccess) return DROPLET_ERR_NOMEM;
    owned.push_back(*q);
    return 0;
  }
  int alloc(const Geo& g) {
    const long long N = g.N;
    const int na = nact(g);
    int rc = 0;
    for (int q = 0; q < J_COUNT && !rc; ++q) {
      int a = -1;
      if (q >= J_U0 && q <= J_U2) a = q - J_U0;
      if (q >= J_FL0 && q <= J_FL2) a = q - J_FL0;
      if (q >= J_AF0 && q <= J_AF2) a = q - J_AF0;
      if (q >= J_US0 && q <= J_US2) a = q - J_US0;
      if (a >= na) continue;
      rc = get(&lam[q], a >= 0 ? nfaces(g, a) : N);
    }
    double** cells[] = {&lA, &lT, &lW, &lP, &lT1, &lW1, &wp, &mu, &bxa, &bmu, &mrbar, &scr1, &scr2};
    for (auto q : cells)
      if (!rc) rc = get(q, N);
    for (int a = 0; a < na && !rc; ++a) rc = get(&lU[a], nfaces(g, a));
    if (!rc) rc = get(&part, RED_BLOCKS * 4);
    if (!rc) rc = get(&acc, AC_COUNT);
    return rc;
  }
  void release() {
    for (auto q : owned) cudaFree(q);
    owned.clear();
  }
  // the state n pointers into a saved state
  void point_state(const Geo& g, const double* s) {
    const long long N = g.N;
    sA = s; sT = s + N; sW = s + 2 * N; sP = s + 3 * N;
    long long o = 4 * N;
    for (int a = 0; a < 3; ++a) {
      sU[a] = a < nact(g) ? s + o : s + 4 * N;
      if (a < nact(g)) o += nfaces(g, a);
    }
  }
};

// Reverse of the step n -> n+1 just re-run from the state w.s*: turns the adjoints of the
// state after the step (w.lA, lT, lW, lP, lU) into those of the state before it, adds
// jweight sum mdot V (the step's share of J) and the parameter adjoints into w.acc.
static int flow_reverse(dctx* x, FlowWork& w, double jweight, int* nc) {
  Geo& g = x->g;
  Phys& p = x->p;
  cudaStream_t st = x->st;
  const long long N = g.N;
  const int na = nact(g);
  const int gc = lin_grid(N);
  const double ADJ_RTOL = 1e-14;
  for (int q = 0; q < J_COUNT; ++q) {
    if (!w.lam[q]) continue;
    int a = -1;
    if (q >= J_U0 && q <= J_U2) a = q - J_U0;
    if (q >= J_FL0 && q <= J_FL2) a = q - J_FL0;
    if (q >= J_AF0 && q <= J_AF2) a = q - J_AF0;
    if (q >= J_US0 && q <= J_US2) a = q - J_US0;
    cudaMemsetAsync(w.lam[q], 0, sizeof(double) * (a >= 0 ? nfaces(g, a) : N), st);
  }
  cudaMemcpyAsync(w.lam[J_ALPHA1], w.lA, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(w.lam[J_P_N], w.lP, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(w.lam[J_DP], w.lP, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(w.lT1, w.lT, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(w.lW1, w.lW, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  L_adj_pin(st, g, p, w.sA, w.sT, w.sW, w.wp);
  FlowIn in;
  in.alpha_n = w.sA; in.T_n = w.sT; in.wp = w.wp; in.p_n = w.sP;
  for (int a = 0; a < 3; ++a) {
    const int aa = a < na ? a : 0;
    in.u[a] = w.sU[aa];
    in.FL[a] = x->FL[aa]; in.AF[a] = x->AF[aa]; in.us[a] = x->us[aa];
  }
  in.astar = x->astar; in.aL = x->aL; in.Rp = x->Rp; in.Rm = x->Rm;
  in.alpha1 = x->alpha; in.rho = x->rho; in.mu = x->mu; in.kc = x->kc; in.cp = x->cp; in.Dm = x->Dm;
  in.mdot = x->mdot; in.rgo = x->rhoG_old; in.rgn = x->rhoG; in.yq = x->yq; in.dp = x->dp; in.xi = x->xi;
  in.adj = x->adj;
  AdjT T;
  for (int q = 0; q < J_COUNT; ++q) T.lam[q] = w.lam[q];
  T.acc = w.acc;
  double* const bc2 = na == 3 ? x->bc[2] : x->bc[0];
  const double* sU2 = na == 3 ? w.sU[2] : w.sU[0];
  const double* us2 = na == 3 ? x->us[2] : x->us[0];
  SolveStats ss;
  int rc;
  // S10: u^{n+1} = u* - dt grad(dp)/rho_f, p^{n+1} = p^n + dp
  L_adjf_correct(st, g, p, in, T, w.lU);
  // S8, S9: the pressure system (symmetric), solved again for the adjoint
  BoxSys bs;
  bs.D = x->bD; bs.b = x->brhs; bs.x = x->bx;
  for (int a = 0; a < 3; ++a) { bs.c[a] = a < na ? x->bc[a] : nullptr; bs.m[a] = g.n[a]; }
  bs.N = N;
  L_poisson_assemble(st, gc, g, p, x->mdot, x->alpha, x->rhoG_old, x->rhoG, w.sU[0], w.sU[1], sU2, x->us[0],
                     x->us[1], us2, x->rho, x->T, x->T, nullptr, w.scr1, x->bD, x->bc[0], x->bc[1], bc2, x->brhs,
                     w.scr2);
  cudaMemcpyAsync(x->brhs, w.lam[J_DP], sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  cudaMemsetAsync(x->bx, 0, sizeof(double) * N, st);
  rc = x->solver.pcg_mg(bs, ADJ_RTOL, 4 * x->cfg.cg_maxit, 0, &ss);
  if ((rc = soft_status(rc, nc))) return rc;
  cudaMemcpyAsync(w.mu, x->bx, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  L_adjf_poisson(st, g, p, in, T, w.mu, x->dp);
  // S7: each velocity component's Helmholtz system
  for (int c = 0; c < na; ++c) {
    int m[3] = {g.n[0], g.n[1], g.n[2]};
    m[c] -= 1;
    const long long nbx = (long long)m[0] * m[1] * m[2];
    BoxSys bm = bs;
    for (int a = 0; a < 3; ++a) bm.m[a] = m[a];
    bm.N = nbx;
    L_mom_assemble(st, lin_grid(nbx), g, p, c, w.sU[0], w.sU[1], sU2, x->rho, x->mu, w.sP, x->alpha, x->xi, x->bD,
                   x->bc[0], x->bc[1], bc2, x->brhs, nullptr);
    cudaMemsetAsync(x->brhs, 0, sizeof(double) * nbx, st);
    L_adjf_box_rhs(st, g, c, w.lam[J_US0 + c], x->brhs, w.lam[J_U0 + c]);
    cudaMemsetAsync(x->bx, 0, sizeof(double) * nbx, st);
    rc = x->solver.pcg_jacobi(bm, ADJ_RTOL, 4 * x->cfg.helm_maxit, &ss);
    if ((rc = soft_status(rc, nc))) return rc;
    cudaMemcpyAsync(w.bmu, x->bx, sizeof(double) * nbx, cudaMemcpyDeviceToDevice, st);
    L_adjf_box_gather(st, g, c, x->us[c], w.bxa);
    L_adjf_mom(st, g, p, in, T, c, w.bmu, w.bxa);
  }
  // rho_G^{n+1} (used by the Stefan source only)
  L_adjf_rhoG(st, g, p, x->T, x->omega, w.lam[J_RGN], w.lT1, w.lW1);
  // S6 species, then the pinned rows' saturation values
  L_scalar_assemble(st, gc, g, p, 1, w.wp, x->rho, x->cp, x->kc, x->Dm, x->mdot, w.sU[0], w.sU[1], sU2, x->alpha,
                    x->yq, 0.0, x->bD, x->bc[0], x->bc[1], bc2, x->brhs, nullptr);
  cudaMemcpyAsync(x->brhs, w.lW1, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  cudaMemsetAsync(x->bx, 0, sizeof(double) * N, st);
  rc = x->solver.pcg_jacobi(bs, ADJ_RTOL, 4 * x->cfg.helm_maxit, &ss);
  if ((rc = soft_status(rc, nc))) return rc;
  cudaMemcpyAsync(w.mu, x->bx, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  L_adjf_scalar(st, g, p, in, T, 1, w.mu, x->omega);
  L_adjf_yq(st, g, p, x->T, x->alpha, w.lam[J_YQ], w.lT1);
  // S5 energy
  L_scalar_assemble(st, gc, g, p, 0, w.sT, x->rho, x->cp, x->kc, x->Dm, x->mdot, w.sU[0], w.sU[1], sU2, x->alpha,
                    x->yq, p.T_amb, x->bD, x->bc[0], x->bc[1], bc2, x->brhs, nullptr);
  cudaMemcpyAsync(x->brhs, w.lT1, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  cudaMemsetAsync(x->bx, 0, sizeof(double) * N, st);
  rc = x->solver.pcg_jacobi(bs, ADJ_RTOL, 4 * x->cfg.helm_maxit, &ss);
  if ((rc = soft_status(rc, nc))) return rc;
  cudaMemcpyAsync(w.mu, x->bx, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  L_adjf_scalar(st, g, p, in, T, 0, w.mu, x->T);
  // S4, S3, S2 with J, S1, S0
  L_adjf_props(st, g, p, in, T);
  L_adjf_fct(st, g, p, in, T);
  L_adjf_source(st, g, p, in, T, x->mraw, x->scal, jweight, w.mrbar, w.part);
  L_adjf_mraw(st, g, p, in, T, w.mrbar);
  L_adj_thermo(st, g, p, w.sA, w.sT, w.wp, x->rhoG_old, w.lam[J_RGO], w.lam[J_WP], w.lam[J_T_N], w.lW);
  cudaMemcpyAsync(w.lA, w.lam[J_ALPHA_N], sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(w.lT, w.lam[J_T_N], sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(w.lP, w.lam[J_P_N], sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  for (int a = 0; a < na; ++a)
    cudaMemcpyAsync(w.lU[a], w.lam[J_U0 + a], sizeof(double) * nfaces(g, a), cudaMemcpyDeviceToDevice, st);
  CKR(cudaGetLastError());
  return 0;
}

// the configurations the flow adjoint differentiates
static bool flow_adjoint_ok(const dctx* x) {
  const droplet_config& cf = x->cfg;
  return cf.physics_mask == (DROPLET_PHYS_EVAP | DROPLET_PHYS_ENERGY | DROPLET_PHYS_SPECIES | DROPLET_PHYS_FLOW) &&
         cf.precision == 0 && cf.eq_model == 0 && cf.const_props_check == 0 && cf.co_max == 0.0 &&
         cf.drho_l_dT == 0.0 && cf.adv_scheme == 0 && cf.fiber == 0 && cf.cp_v == cf.cp_g;
}

static int adjoint_flow(droplet_ctx* cc, int n_steps, int ckpt_every, double* J, double* dJ_dTamb, double* dJ_dDg,
                        double* dJ_dT0, size_t nT0) {
  dctx* x = cc->d[0];
  if (!flow_adjoint_ok(x) || x->step != 0) return DROPLET_ERR_ARG;
  Geo& g = x->g;
  Phys& p = x->p;
  const long long N = g.N;
  if (dJ_dT0 && nT0 != (size_t)N) return DROPLET_ERR_SIZE;
  cudaStream_t st = x->st;
  CKR(cudaStreamSynchronize(cc->st));
  CKR(cudaStreamSynchronize(st));
  const int nseg = (n_steps + ckpt_every - 1) / ckpt_every;
  const long long S = flow_state_size(x);
  double *ck = nullptr, *seg = nullptr, *fin = nullptr;
  FlowWork w;
  auto cleanup = [&]() { cudaFree(ck); cudaFree(seg); cudaFree(fin); w.release(); };
  if (cudaMalloc(&ck, sizeof(double) * S * nseg) != cudaSuccess ||
      cudaMalloc(&seg, sizeof(double) * S * (ckpt_every + 1)) != cudaSuccess ||
      cudaMalloc(&fin, sizeof(double) * S) != cudaSuccess || w.alloc(g)) {
    cleanup();
    return DROPLET_ERR_NOMEM;
  }
  cudaMemsetAsync(w.acc, 0, sizeof(double) * AC_COUNT, st);
  const double jweight = (g.axisym ? 2.0 * M_PI : 1.0) / n_steps;
  int nc = 0, rc = 0;
  for (int n = 0; n < n_steps && !rc; ++n) {
    if (n % ckpt_every == 0) flow_save(x, ck + S * (n / ckpt_every));
    rc = flow_step_alone(x, &nc);
    L_acc_J(st, x->scal, jweight, w.acc);
  }
  flow_save(x, fin);
  CKR(cudaStreamSynchronize(st));
  double host_acc[AC_COUNT];
  CKR(cudaMemcpy(host_acc, w.acc, sizeof(double) * AC_COUNT, cudaMemcpyDeviceToHost));
  *J = host_acc[AC_J];
  if (!rc && (dJ_dTamb || dJ_dDg || dJ_dT0)) {
    const int na = nact(g);
    cudaMemsetAsync(w.lA, 0, sizeof(double) * N, st);
    cudaMemsetAsync(w.lT, 0, sizeof(double) * N, st);
    cudaMemsetAsync(w.lW, 0, sizeof(double) * N, st);
    cudaMemsetAsync(w.lP, 0, sizeof(double) * N, st);
    for (int a = 0; a < na; ++a) cudaMemsetAsync(w.lU[a], 0, sizeof(double) * nfaces(g, a), st);
    for (int sgi = nseg - 1; sgi >= 0 && !rc; --sgi) {
      const int n0 = sgi * ckpt_every, n1 = n0 + ckpt_every < n_steps ? n0 + ckpt_every : n_steps;
      flow_load(x, ck + S * sgi);
      for (int n = n0; n < n1 && !rc; ++n) {
        flow_save(x, seg + S * (n - n0));
        if (n + 1 < n1) rc = flow_step_alone(x, &nc);
      }
      for (int n = n1 - 1; n >= n0 && !rc; --n) {
        const double* sn = seg + S * (n - n0);
        flow_load(x, sn);
        rc = flow_step_alone(x, &nc);   // leaves step n's intermediates and state n+1
        if (rc) break;
        w.point_state(g, sn);
        rc = flow_reverse(x, w, jweight, &nc);
      }
    }
    if (!rc) {
      L_adj_tamb(st, g, p, w.lT, w.part, w.acc);
      CKR(cudaStreamSynchronize(st));
      CKR(cudaMemcpy(host_acc, w.acc, sizeof(double) * AC_COUNT, cudaMemcpyDeviceToHost));
      if (dJ_dDg) *dJ_dDg = host_acc[AC_DGAS] * (1.0e5 / x->cfg.P);
      if (dJ_dTamb) *dJ_dTamb = host_acc[AC_TAMB] + host_acc[AC_TAMB_BC];
      if (dJ_dT0) CKR(cudaMemcpy(dJ_dT0, w.lT, sizeof(double) * N, cudaMemcpyDeviceToHost));
    }
  }
  flow_load(x, fin);
  CKR(cudaStreamSynchronize(st));
  cleanup();
  {
    const double tn = n_steps * p.dt;
    CKR(cudaMemcpy(x->scal + SC_TIME, &tn, sizeof(double), cudaMemcpyHostToDevice));
  }
  x->step = n_steps;
  if (rc) return rc;
  return nc ? DROPLET_ERR_NOT_CONVERGED : 0;
}

extern "C" int droplet_adjoint_vjp(droplet_ctx* cc, const double* lam_next, double* lam_prev, size_t n,
                                   double mdot_weight, double* dpar) {
  if (!cc || cc->d.size() != 1 || !lam_next || !lam_prev) return DROPLET_ERR_ARG;
  dctx* x = cc->d[0];
  if (!flow_adjoint_ok(x)) return DROPLET_ERR_ARG;
  const long long S = flow_state_size(x);
  if (n != (size_t)S) return DROPLET_ERR_SIZE;
  Geo& g = x->g;
  const long long N = g.N;
  const int na = nact(g);
  cudaStream_t st = x->st;
  CKR(cudaStreamSynchronize(cc->st));
  double* s0 = nullptr;
  FlowWork w;
  if (cudaMalloc(&s0, sizeof(double) * S) != cudaSuccess || w.alloc(g)) {
    cudaFree(s0);
    w.release();
    return DROPLET_ERR_NOMEM;
  }
  cudaMemsetAsync(w.acc, 0, sizeof(double) * AC_COUNT, st);
  flow_save(x, s0);
  // the adjoint of the state after the step, in the packed layout
  double* dst[8] = {w.lA, w.lT, w.lW, w.lP, w.lU[0], w.lU[1], w.lU[2], nullptr};
  long long sz[7] = {N, N, N, N, na > 0 ? nfaces(g, 0) : 0, nfaces(g, 1), na == 3 ? nfaces(g, 2) : 0};
  long long o = 0;
  for (int q = 0; q < 4 + na; ++q) {
    CKR(cudaMemcpyAsync(dst[q], lam_next + o, sizeof(double) * sz[q], cudaMemcpyHostToDevice, st));
    o += sz[q];
  }
  int nc = 0;
  flow_load(x, s0);
  int rc = flow_step_alone(x, &nc);
  if (!rc) {
    w.point_state(g, s0);
    rc = flow_reverse(x, w, mdot_weight * (g.axisym ? 2.0 * M_PI : 1.0), &nc);
  }
  if (!rc) {
    CKR(cudaStreamSynchronize(st));
    o = 0;
    for (int q = 0; q < 4 + na; ++q) {
      CKR(cudaMemcpy(lam_prev + o, dst[q], sizeof(double) * sz[q], cudaMemcpyDeviceToHost));
      o += sz[q];
    }
    double host_acc[AC_COUNT];
    CKR(cudaMemcpy(host_acc, w.acc, sizeof(double) * AC_COUNT, cudaMemcpyDeviceToHost));
    if (dpar) {
      dpar[0] = host_acc[AC_TAMB_BC];
      dpar[1] = host_acc[AC_DGAS] * (1.0e5 / x->cfg.P);
    }
  }
  cudaFree(s0);
  w.release();
  ++x->step;
  if (rc) return rc;
  return nc ? DROPLET_ERR_NOT_CONVERGED : 0;
}

extern "C" int droplet_adjoint_check(droplet_ctx* cc, double* rel, int nrel) {
  if (!cc || cc->d.size() != 1 || !rel || nrel < CHK_COUNT) return DROPLET_ERR_ARG;
  dctx* x = cc->d[0];
  if (!flow_adjoint_ok(x)) return DROPLET_ERR_ARG;
  Geo& g = x->g;
  Phys& p = x->p;
  const long long N = g.N;
  const int na = nact(g);
  cudaStream_t st = x->st;
  CKR(cudaStreamSynchronize(cc->st));
  const long long S = flow_state_size(x);
  double* s0 = nullptr;
  double* wp = nullptr;
  double* scr = nullptr;
  unsigned long long* chk = nullptr;
  auto cleanup = [&]() { cudaFree(s0); cudaFree(wp); cudaFree(scr); cudaFree(chk); };
  if (cudaMalloc(&s0, sizeof(double) * S) != cudaSuccess || cudaMalloc(&wp, sizeof(double) * N) != cudaSuccess ||
      cudaMalloc(&scr, sizeof(double) * 2 * N) != cudaSuccess ||
      cudaMalloc(&chk, sizeof(unsigned long long) * 2 * CHK_COUNT) != cudaSuccess) {
    cleanup();
    return DROPLET_ERR_NOMEM;
  }
  cudaMemsetAsync(chk, 0, sizeof(unsigned long long) * 2 * CHK_COUNT, st);
  flow_save(x, s0);
  int nc = 0;
  flow_load(x, s0);
  int rc = flow_step_alone(x, &nc);
  if (!rc) {
    const double* sA = s0;
    const double* sT = s0 + N;
    const double* sW = s0 + 2 * N;
    const double* sP = s0 + 3 * N;
    const double* sU[3];
    long long o = 4 * N;
    for (int a = 0; a < 3; ++a) {
      sU[a] = a < na ? s0 + o : s0 + 4 * N;
      if (a < na) o += nfaces(g, a);
    }
    L_adj_pin(st, g, p, sA, sT, sW, wp);
    FlowIn in;
    in.alpha_n = sA; in.T_n = sT; in.wp = wp; in.p_n = sP;
    for (int a = 0; a < 3; ++a) {
      const int aa = a < na ? a : 0;
      in.u[a] = sU[aa];
      in.FL[a] = x->FL[aa]; in.AF[a] = x->AF[aa]; in.us[a] = x->us[aa];
    }
    in.astar = x->astar; in.aL = x->aL; in.Rp = x->Rp; in.Rm = x->Rm;
    in.alpha1 = x->alpha; in.rho = x->rho; in.mu = x->mu; in.kc = x->kc; in.cp = x->cp; in.Dm = x->Dm;
    in.mdot = x->mdot; in.rgo = x->rhoG_old; in.rgn = x->rhoG; in.yq = x->yq; in.dp = x->dp; in.xi = x->xi;
    in.adj = x->adj;
    double* const bc2 = na == 3 ? x->bc[2] : x->bc[0];
    double* const C[3] = {x->bc[0], x->bc[1], na == 3 ? x->bc[2] : nullptr};
    L_chk_cells(st, g, p, in, x->mraw, chk);
    L_chk_faces(st, g, p, in, x->u, chk);
    for (int mode = 0; mode < 2; ++mode) {
      L_scalar_assemble(st, lin_grid(N), g, p, mode, mode == 0 ? sT : wp, x->rho, x->cp, x->kc, x->Dm, x->mdot, sU[0],
                        sU[1], sU[2], x->alpha, x->yq, mode == 0 ? p.T_amb : 0.0, x->bD, x->bc[0], x->bc[1], bc2,
                        x->brhs, nullptr);
      L_chk_rows(st, g, p, in, mode, x->bD, C, x->brhs, chk);
    }
    L_poisson_assemble(st, lin_grid(N), g, p, x->mdot, x->alpha, x->rhoG_old, x->rhoG, sU[0], sU[1], sU[2], x->us[0],
                       x->us[1], na == 3 ? x->us[2] : x->us[0], x->rho, x->T, x->T, nullptr, scr, x->bD, x->bc[0],
                       x->bc[1], bc2, x->brhs, scr + N);
    L_chk_rows(st, g, p, in, 2, x->bD, C, x->brhs, chk);
    for (int c = 0; c < na; ++c) {
      int m[3] = {g.n[0], g.n[1], g.n[2]};
      m[c] -= 1;
      L_mom_assemble(st, lin_grid((long long)m[0] * m[1] * m[2]), g, p, c, sU[0], sU[1], sU[2], x->rho, x->mu, sP,
                     x->alpha, x->xi, x->bD, x->bc[0], x->bc[1], bc2, x->brhs, nullptr);
      L_chk_rows(st, g, p, in, 3 + c, x->bD, C, x->brhs, chk);
    }
    CKR(cudaStreamSynchronize(st));
    unsigned long long h[2 * CHK_COUNT];
    CKR(cudaMemcpy(h, chk, sizeof(h), cudaMemcpyDeviceToHost));
    for (int q = 0; q < CHK_COUNT; ++q) {
      double d, r;
      memcpy(&d, &h[2 * q], sizeof(double));
      memcpy(&r, &h[2 * q + 1], sizeof(double));
      rel[q] = r > 0.0 ? d / r : d;
    }
  }
  cleanup();
  ++x->step;
  if (rc) return rc;
  return nc ? DROPLET_ERR_NOT_CONVERGED : 0;
}

// ---------------------------------------------------------------- checkpoint / resume
// (format 5: the configuration carries the fibre field)
static const char kMagic[8] = {'D', 'R', 'O', 'P', 'C', 'K', 'P', '5'};

// the checkpointed fields: the state, the history of the extrapolated guesses, and the
// liquid's expansion term of the last step (a temperature-dependent liquid density only)
constexpr int NCKPT = 14;
static int state_fields(dctx* x, double* f[NCKPT], long long n[NCKPT]) {
  double* fs[NCKPT] = {x->alpha, x->T, x->omega, x->pr, x->rhoG, x->u[0], x->u[1], x->u[2],
                       x->hT, x->hW, x->hu[0], x->hu[1], x->hu[2], x->expand};
  for (int q = 0; q < NCKPT; ++q) {
    f[q] = fs[q];
    const int fa = q >= 10 && q < 13 ? q - 10 : q - 5;
    const bool cell = q < 5 || q == 8 || q == 9 || q == 13;
    n[q] = fs[q] ? (cell ? x->g.N : nfaces(x->g, fa)) : 0;
  }
  return 0;
}

extern "C" int droplet_save(droplet_ctx* c, const char* path) {
  if (!c || !path) return DROPLET_ERR_ARG;
  CKR(cudaStreamSynchronize(c->st));
  FILE* fp = fopen(path, "wb");
  if (!fp) return DROPLET_ERR_IO;
  long long nd = (long long)c->d.size();
  bool ok = fwrite(kMagic, 1, 8, fp) == 8 && fwrite(&nd, sizeof(nd), 1, fp) == 1;
  std::vector<double> host;
  for (auto x : c->d) {
    if (!ok) break;
    CKR(cudaStreamSynchronize(x->st));
    CKR(cudaMemcpy(x->hscal, x->scal, sizeof(double) * SC_COUNT, cudaMemcpyDeviceToHost));
    ok = fwrite(&x->cfg, sizeof(droplet_config), 1, fp) == 1 && fwrite(&x->hscal[SC_TIME], sizeof(double), 1, fp) == 1 &&
         fwrite(&x->step, sizeof(long long), 1, fp) == 1 && fwrite(x->hscal, sizeof(double), SC_COUNT, fp) == SC_COUNT;
    double* f[NCKPT];
    long long n[NCKPT];
    state_fields(x, f, n);
    for (int q = 0; q < NCKPT && ok; ++q) {
      if (!n[q]) continue;
      host.resize((size_t)n[q]);
      if (cudaMemcpy(host.data(), f[q], sizeof(double) * n[q], cudaMemcpyDeviceToHost) != cudaSuccess) { fclose(fp); return DROPLET_ERR_CUDA; }
      ok = fwrite(host.data(), sizeof(double), (size_t)n[q], fp) == (size_t)n[q];
    }
  }
  if (fclose(fp) != 0) ok = false;
  return ok ? 0 : DROPLET_ERR_IO;
}

extern "C" int droplet_load(droplet_ctx* c, const char* path) {
  if (!c || !path) return DROPLET_ERR_ARG;
  CKR(cudaStreamSynchronize(c->st));
  FILE* fp = fopen(path, "rb");
  if (!fp) return DROPLET_ERR_IO;
  char mg[8];
  long long nd = 0;
  if (fread(mg, 1, 8, fp) != 8 || memcmp(mg, kMagic, 8) != 0 || fread(&nd, sizeof(nd), 1, fp) != 1) { fclose(fp); return DROPLET_ERR_IO; }
  if (nd != (long long)c->d.size()) { fclose(fp); return DROPLET_ERR_ARG; }
  std::vector<double> host;
  for (auto x : c->d) {
    droplet_config cf;
    double t;
    long long step;
    if (fread(&cf, sizeof(cf), 1, fp) != 1 || fread(&t, sizeof(t), 1, fp) != 1 || fread(&step, sizeof(step), 1, fp) != 1 ||
        fread(x->hscal, sizeof(double), SC_COUNT, fp) != SC_COUNT) { fclose(fp); return DROPLET_ERR_IO; }
    if (memcmp(&cf, &x->cfg, sizeof(cf)) != 0) { fclose(fp); return DROPLET_ERR_ARG; }
    CKR(cudaStreamSynchronize(x->st));
    double* f[NCKPT];
    long long n[NCKPT];
    state_fields(x, f, n);
    for (int q = 0; q < NCKPT; ++q) {
      if (!n[q]) continue;
      host.resize((size_t)n[q]);
      if (fread(host.data(), sizeof(double), (size_t)n[q], fp) != (size_t)n[q]) { fclose(fp); return DROPLET_ERR_IO; }
      if (cudaMemcpy(f[q], host.data(), sizeof(double) * n[q], cudaMemcpyHostToDevice) != cudaSuccess) { fclose(fp); return DROPLET_ERR_CUDA; }
    }
    if (cudaMemcpy(x->scal, x->hscal, sizeof(double) * SC_COUNT, cudaMemcpyHostToDevice) != cudaSuccess) { fclose(fp); return DROPLET_ERR_CUDA; }
    (void)t;   // the clock is restored with the device scalars
    x->step = step;
    // the saved rho_G is rho_gas(T, omega) of the saved state: S0 may reuse it
    if (cudaMemset(x->dirty, 0, sizeof(int)) != cudaSuccess) { fclose(fp); return DROPLET_ERR_CUDA; }
  }
  fclose(fp);
  return 0;
}

extern "C" int droplet_box_solve(const int m[3], const double* D, const double* c0, const double* c1,
                                 const double* c2, const double* b, double* x, double rtol, int maxit,
                                 void* cuda_stream, int* its, double* relres) {
  if (!m || !D || !c0 || !c1 || !b || !x || maxit < 1 || !(rtol > 0.0)) return DROPLET_ERR_ARG;
  if (m[0] < 1 || m[1] < 1 || m[2] < 1 || (m[2] > 1 && !c2)) return DROPLET_ERR_ARG;
  long long N = (long long)m[0] * m[1] * m[2];
  Solver sv;
  int rc = sv.setup(N, (cudaStream_t)cuda_stream);
  if (rc) { sv.release(); return rc; }
  BoxSys bs;
  for (int a = 0; a < 3; ++a) bs.m[a] = m[a];
  bs.N = N;
  bs.D = (double*)D;
  bs.c[0] = (double*)c0;
  bs.c[1] = (double*)c1;
  bs.c[2] = m[2] > 1 ? (double*)c2 : nullptr;
  bs.b = (double*)b;
  bs.x = x;
  SolveStats ss;
  rc = sv.pcg_jacobi(bs, rtol, maxit, &ss);
  sv.release();
  if (its) *its = ss.its;
  if (relres) *relres = ss.relres;
  return rc;
}
