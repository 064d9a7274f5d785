// Hand-written discrete adjoint of one time step of the droplet method without
// flow (evaporation flux with the K normalisation of Eq. alphafunction, alpha
// source of Eq. alphasource, energy Eq. Teqn, species Eq. speciesequation with
// the liquid rows pinned to the Raoult saturation value, gas density of
// Eq. densitygas).  Discrete branch decisions of the forward step (interface
// cells, adjacent gas cells, the mdot cap, alpha clipping, the pinned set) are
// held fixed.  FP64.
//
// Notation: for step n -> n+1 the forward re-run leaves alpha^{n+1}, T^{n+1},
// omega^{n+1}, rho_G^n, mdot, m_raw, alpha*, adj and the mixture properties in
// the context's arrays; the state of step n is passed separately.  The adjoint
// of the state after the step (aA, aT, aW) is turned into that of the state
// before it, and the derivative with respect to the gas diffusivity is
// accumulated in acc[AC_DGAS].
#include "common.cuh"
#include "kernels.h"

namespace dg {

__device__ __forceinline__ double harm_(double x, double y) { return 2.0 * x * y / (x + y); }
// d/dx of the harmonic mean 2xy/(x+y)
__device__ __forceinline__ double dharm_dx(double x, double y) { return 2.0 * y * y / ((x + y) * (x + y)); }

// neighbour of cell (i,j,k) across face `side` of axis a, -1 when outside the domain
__device__ __forceinline__ long long nbr(const Geo& g, int i, int j, int k, int a, int side) {
  int q[3] = {i, j, k};
  q[a] += side ? 1 : -1;
  if (q[a] < 0 || q[a] >= g.n[a]) return -1;
  return cidx(g, q[0], q[1], q[2]);
}
// area of the face of cell (i,..) on side `side` of axis a
__device__ __forceinline__ double face_area_side(const Geo& g, int a, int i, int side) {
  if (a == 0) return faceA(g, 0, i + side);
  return faceA(g, a, i);
}

// omega' = omega with the liquid cells (alpha >= 1/2) set to Y_eq(T)
__global__ void k_adj_pin(Geo g, Phys p, const double* alpha, const double* T, const double* omega, double* wp) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  wp[id] = alpha[id] >= 0.5 ? Y_eq(p, T[id], nullptr) : omega[id];
}

// right-hand side of an adjoint solve: the state adjoint on free rows, 0 on pinned rows
__global__ void k_adj_rhs(Geo g, const double* abar, const double* alpha_new, int pinned_rows, double* rhs, double* x) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  bool pin = pinned_rows && alpha_new[id] >= 0.5;
  rhs[id] = pin ? 0.0 : abar[id];
  x[id] = 0.0;
}

// Species coefficient adjoints.  bW: adjoint solution on the free rows.  Writes
// Tn1bar (adjoint of T^{n+1} from the pinned rows, plus aT), wpbar (adjoint of omega'),
// rhobar and Dbar (adjoints of the mixture rho and D).
__global__ void k_adj_species(Geo g, Phys p, const double* bW, const double* aW, const double* aT,
                              const double* alpha_new, const double* wp, const double* wn1, const double* Tn1,
                              const double* rho, const double* D, double* Tn1bar, double* wpbar, double* rhobar,
                              double* Dbar) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  int i, j, k;
  decomp(id, g.n[0], g.n[1], i, j, k);
  int na = nact(g);
  double V = cellV(g, i);
  bool pin = alpha_new[id] >= 0.5;
  double gP = rho[id] * D[id];
  double gbar = 0.0, tb = aT[id], wpb = 0.0, rb = 0.0;
  double bP = bW[id];
  double pinned_b = aW[id];
  for (int a = 0; a < na; ++a)
    for (int side = 0; side < 2; ++side) {
      long long q = nbr(g, i, j, k, a, side);
      if (q < 0) continue;
      bool qpin = alpha_new[q] >= 0.5;
      if (pin && qpin) continue;
      double gQ = rho[q] * D[q];
      double A = face_area_side(g, a, i, side) * g.ih[a];
      double c = harm_(gP, gQ) * A;
      if (pin) {
        // free neighbour Q couples to this pinned value: d(rhs_Q)/d(yq_P) = c
        pinned_b += c * bW[q];
      }
      double cbar = -(pin ? 0.0 : bP) * (wn1[id] - wn1[q]) - (qpin ? 0.0 : bW[q]) * (wn1[q] - wn1[id]);
      gbar += cbar * dharm_dx(gP, gQ) * A;
    }
  if (pin) {
    tb += pinned_b * dYeq_dT(p, Tn1[id]);
  } else {
    rb += bP * V * (wp[id] - wn1[id]) * p.idt;
    wpb = bP * rho[id] * V * p.idt;
  }
  rb += gbar * D[id];
  Tn1bar[id] = tb;
  wpbar[id] = wpb;
  rhobar[id] = rb;
  Dbar[id] = gbar * rho[id];
}

// Energy coefficient adjoints.  bT: adjoint solution.  Writes Tnbar (adjoint of T^n so far),
// adds to rhobar, writes kbar, cpbar, mdbar (adjoint of mdot from the source -mdot L V).
__global__ void k_adj_energy(Geo g, Phys p, const double* bT, const double* Tn, const double* Tn1, const double* rho,
                             const double* cp, const double* kc, double* Tnbar, double* rhobar, double* kbar,
                             double* cpbar, double* mdbar) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  int i, j, k;
  decomp(id, g.n[0], g.n[1], i, j, k);
  int na = nact(g);
  double V = cellV(g, i);
  double bP = bT[id];
  double rcp = rho[id] * cp[id];
  Tnbar[id] = bP * rcp * V * p.idt;
  double rcpbar = bP * V * (Tn[id] - Tn1[id]) * p.idt;
  mdbar[id] = -bP * p.Lv * V;
  double kb = 0.0;
  for (int a = 0; a < na; ++a)
    for (int side = 0; side < 2; ++side) {
      long long q = nbr(g, i, j, k, a, side);
      if (q < 0) continue;
      double A = face_area_side(g, a, i, side) * g.ih[a];
      double cbar = -(bP - bT[q]) * (Tn1[id] - Tn1[q]);
      kb += cbar * dharm_dx(kc[id], kc[q]) * A;
    }
  kbar[id] = kb;
  rhobar[id] += rcpbar * cp[id];
  cpbar[id] = rcpbar * rho[id];
}

// Mixture properties, clipping, alpha source, J and the mdot cap.  Writes the adjoint of
// alpha^n so far (aAn), of rho_G^n (rgbar), the final mdot adjoint (mdbar, 0 where capped)
// and block sums of: D_gas adjoint, sum(mdbar f m_raw) (= K bar), S1, S2.
__global__ void k_adj_props_source(Geo g, Phys p, const double* aA, const double* alpha_n, const double* alpha_new,
                                   const double* astar, const double* rgn, const double* mraw, const double* scal,
                                   const double* rhobar, const double* kbar, const double* cpbar, const double* Dbar,
                                   double jweight, double* aAn, double* rgbar, double* mdbar, double* part) {
  double acc[4] = {0, 0, 0, 0};
  double K = scal[SC_K];
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < g.N; id += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    decomp(id, g.n[0], g.n[1], i, j, k);
    double V = cellV(g, i);
    double an1 = alpha_new[id];
    // properties at alpha^{n+1}, rho_G^n
    double abar = aA[id] + rhobar[id] * (p.rho_l - rgn[id]) + kbar[id] * (p.k_l - p.k_g) +
                  cpbar[id] * (p.cp_l - p.cp_g) + Dbar[id] * (p.D_l - p.D_gas);
    rgbar[id] = rhobar[id] * (1.0 - an1);
    acc[0] += Dbar[id] * (1.0 - an1);
    // clipping: the clipped value is a constant
    double as = astar[id];
    double asbar = (as == an1) ? abar : 0.0;
    // alpha* = alpha - dt mdot / rho_L; J = w sum mdot V / nsteps
    double an = alpha_n[id];
    double md = mdbar[id] + jweight * V - p.dt * asbar / p.rho_l;
    double aAn_v = asbar;
    double f = sqrt(an * (1.0 - an));
    double m_unc = (K == 0.0) ? 0.0 : K * f * mraw[id];
    double cap = p.rho_l * an * p.idt;
    if (m_unc > cap) {
      aAn_v += md * p.rho_l * p.idt;
      md = 0.0;
    }
    mdbar[id] = md;
    aAn[id] = aAn_v;
    acc[1] += md * f * mraw[id];
    acc[2] += mraw[id] * V;
    acc[3] += f * mraw[id] * V;
  }
  block_sum_store<4>(acc, part);
}

// K = S1/S2 and mdot = K f m_raw: adjoint of m_raw and the f(alpha) terms of alpha^n
__global__ void k_adj_K(Geo g, Phys p, const double* part, int nblk, const double* alpha_n, const double* mraw,
                        const double* scal, const double* mdbar, double* mrbar, double* aAn, double* acc_out) {
  __shared__ double sums[4];
  for (int q = 0; q < 4; ++q) {
    double v = block_sum_partials(part + q * nblk, nblk);
    if (threadIdx.x == 0) sums[q] = v;
    __syncthreads();
  }
  double K = scal[SC_K];
  double Kbar = sums[1], S1 = sums[2], S2 = sums[3];
  if (blockIdx.x == 0 && threadIdx.x == 0) acc_out[AC_DGAS] += sums[0];
  double S1bar = 0.0, S2bar = 0.0;
  if (K != 0.0 && S2 != 0.0) {
    S1bar = Kbar / S2;
    S2bar = -Kbar * K / S2;
  }
  (void)S1;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < g.N; id += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    decomp(id, g.n[0], g.n[1], i, j, k);
    double V = cellV(g, i);
    double an = alpha_n[id];
    double f = sqrt(an * (1.0 - an));
    double fp = (an > 0.0 && an < 1.0) ? (1.0 - 2.0 * an) / (2.0 * f) : 0.0;   // f' (0 at alpha = 0, 1)
    double mr = mraw[id];
    double md = mdbar[id];
    mrbar[id] = md * K * f + S1bar * V + S2bar * f * V;
    aAn[id] += md * K * fp * mr + S2bar * fp * mr * V;
  }
}

// adjoint of omega' or alpha at a (possibly ghost) cell index of the central differences
__device__ __forceinline__ void add_ghost(const Geo& g, double* bar, int i, int j, int k, double v, bool alpha_rule) {
  int q[3] = {i, j, k};
  for (int a = 0; a < 3; ++a) {
    if (q[a] < 0 || q[a] >= g.n[a]) {
      int side = q[a] < 0 ? 0 : 1;
      int kind = bc_of(g, a, side);
      // alpha: 0 outside every boundary but the axis (mirror); omega without flow: zero gradient / mirror
      if (alpha_rule && kind != BC_AXIS) return;
      q[a] = side ? g.n[a] - 1 : 0;
      break;
    }
  }
  atomicAdd(bar + cidx(g, q[0], q[1], q[2]), v);
}

// m_raw_P = G_Q sum_a g_aP d_a omega'_Q (no flow), G = rho D at the adjacent cell Q:
// scatter into alpha^n (g and G), omega' (gradient at Q), rho_G^n (G) and D_gas (G)
__global__ void k_adj_evap(Geo g, Phys p, const double* alpha_n, const double* wp, const double* rgn, const int* adj,
                           const double* mrbar, double* aAn, double* wpbar, double* rgbar, double* part) {
  double dacc[1] = {0.0};
  int na = nact(g);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < g.N; id += (long long)gridDim.x * blockDim.x) {
    int qid = adj[id];
    double mb = mrbar[id];
    if (qid < 0 || mb == 0.0) continue;
    int i, j, k, qi, qj, qk;
    decomp(id, g.n[0], g.n[1], i, j, k);
    decomp(qid, g.n[0], g.n[1], qi, qj, qk);
    double gr[3], gw[3];
    int ci[3] = {i, j, k}, cq[3] = {qi, qj, qk};
    for (int a = 0; a < 3; ++a) {
      gr[a] = gw[a] = 0.0;
      if (a >= na) continue;
      int pp[3] = {i, j, k}, pm[3] = {i, j, k}, qp[3] = {qi, qj, qk}, qm[3] = {qi, qj, qk};
      pp[a] += 1; pm[a] -= 1; qp[a] += 1; qm[a] -= 1;
      gr[a] = (cellg(g, alpha_n, pp[0], pp[1], pp[2], R_ALPHA, 0, 0, 0, 0) -
               cellg(g, alpha_n, pm[0], pm[1], pm[2], R_ALPHA, 0, 0, 0, 0)) * (0.5 * g.ih[a]);
      gw[a] = (cellg(g, wp, qp[0], qp[1], qp[2], R_ZG, 0, 0, 0, 0) -
               cellg(g, wp, qm[0], qm[1], qm[2], R_ZG, 0, 0, 0, 0)) * (0.5 * g.ih[a]);
    }
    (void)ci; (void)cq;
    double aQ = alpha_n[qid], rgQ = rgn[qid];
    double rhoQ = aQ * p.rho_l + (1.0 - aQ) * rgQ;
    double DQ = aQ * p.D_l + (1.0 - aQ) * p.D_gas;
    double G = rhoQ * DQ;
    double sgw = 0.0;
    for (int a = 0; a < na; ++a) sgw += gr[a] * gw[a];
    double Gbar = mb * sgw;
    atomicAdd(aAn + qid, Gbar * ((p.rho_l - rgQ) * DQ + rhoQ * (p.D_l - p.D_gas)));
    atomicAdd(rgbar + qid, Gbar * (1.0 - aQ) * DQ);
    dacc[0] += Gbar * rhoQ * (1.0 - aQ);
    for (int a = 0; a < na; ++a) {
      double gbar = mb * G * gw[a] * (0.5 * g.ih[a]);
      double wbar = mb * G * gr[a] * (0.5 * g.ih[a]);
      int pp[3] = {i, j, k}, pm[3] = {i, j, k}, qp[3] = {qi, qj, qk}, qm[3] = {qi, qj, qk};
      pp[a] += 1; pm[a] -= 1; qp[a] += 1; qm[a] -= 1;
      add_ghost(g, aAn, pp[0], pp[1], pp[2], gbar, true);
      add_ghost(g, aAn, pm[0], pm[1], pm[2], -gbar, true);
      add_ghost(g, wpbar, qp[0], qp[1], qp[2], wbar, false);
      add_ghost(g, wpbar, qm[0], qm[1], qm[2], -wbar, false);
    }
  }
  block_sum_store<1>(dacc, part);
}

__global__ void k_adj_acc(const double* part, int nblk, double* acc_out) {
  double v = block_sum_partials(part, nblk);
  if (threadIdx.x == 0) acc_out[AC_DGAS] += v;
}

// rho_G^n = P / (R T m(omega')), omega' = pin(omega, T): adjoints of T^n and omega^n
__global__ void k_adj_thermo(Geo g, Phys p, const double* alpha_n, const double* Tn, const double* wp,
                             const double* rgn, const double* rgbar, const double* wpbar, double* Tnbar, double* aW) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  double T = Tn[id], w = wp[id], R = rgn[id];
  double m = w / p.M_l + (1.0 - w) / p.M_g;
  double rb = rgbar[id];
  double tb = Tnbar[id] - rb * R / T;
  double wb = wpbar[id] - rb * R * (1.0 / p.M_l - 1.0 / p.M_g) / m;
  if (alpha_n[id] >= 0.5) {
    tb += wb * dYeq_dT(p, T);
    aW[id] = 0.0;
  } else {
    aW[id] = wb;
  }
  Tnbar[id] = tb;
}

// J += weight * sum(mdot V) of the step just taken
__global__ void k_acc_J(const double* scal, double weight, double* acc_out) {
  acc_out[AC_J] += weight * scal[SC_SUM_MDOT_V];
}

// dJ/dT_amb = sum_P dJ/dT0_P dT0_P/dT_amb through the initial temperature of Sec. 3.3:
// T0 = (T_amb + (T_drop - T_amb) w(r)) (1 + T_perturb u_P)
__global__ void k_adj_tamb(Geo g, Phys p, const double* T0bar, double* part) {
  double acc[1] = {0.0};
  int na = nact(g);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < g.N; id += (long long)gridDim.x * blockDim.x) {
    int q[3];
    decomp(id, g.n[0], g.n[1], q[0], q[1], q[2]);
    double d2 = 0.0;
    for (int a = 0; a < na; ++a) {
      double x = (q[a] + 0.5) * g.h[a] - p.xc[a];
      d2 = d2 + x * x;
    }
    double r = sqrt(d2), rs = 0.5 * p.D0, Rf = 2.0 * p.D0;
    double w = (1.0 / fmax(r, rs) - 1.0 / Rf) / (1.0 / rs - 1.0 / Rf);
    w = fmin(1.0, fmax(0.0, w));
    double fac = 1.0 - w;
    if (p.T_perturb != 0.0) {
      unsigned long long z = (p.seed ^ (unsigned long long)id) + 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z = z ^ (z >> 31);
      double u = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
      fac *= 1.0 + p.T_perturb * u;
    }
    acc[0] += T0bar[id] * fac;
  }
  block_sum_store<1>(acc, part);
}

__global__ void k_adj_tamb_fin(const double* part, int nblk, double* acc_out) {
  double v = block_sum_partials(part, nblk);
  if (threadIdx.x == 0) acc_out[AC_TAMB] = v;
}

// ---------------------------------------------------------------- host launchers
void L_acc_J(cudaStream_t st, const double* scal, double weight, double* acc_out) {
  ++g_launches, k_acc_J<<<1, 1, 0, st>>>(scal, weight, acc_out);
}
void L_adj_tamb(cudaStream_t st, const Geo& g, const Phys& p, const double* T0bar, double* part, double* acc_out) {
  int nb = red_grid(g.N);
  ++g_launches, k_adj_tamb<<<nb, TPB, 0, st>>>(g, p, T0bar, part);
  ++g_launches, k_adj_tamb_fin<<<1, TPB, 0, st>>>(part, nb, acc_out);
}
void L_adj_pin(cudaStream_t st, const Geo& g, const Phys& p, const double* alpha, const double* T,
               const double* omega, double* wp) {
  ++g_launches, k_adj_pin<<<lin_grid(g.N), TPB, 0, st>>>(g, p, alpha, T, omega, wp);
}
void L_adj_rhs(cudaStream_t st, const Geo& g, const double* abar, const double* alpha_new, int pinned_rows,
               double* rhs, double* x) {
  ++g_launches, k_adj_rhs<<<lin_grid(g.N), TPB, 0, st>>>(g, abar, alpha_new, pinned_rows, rhs, x);
}
void L_adj_species(cudaStream_t st, const Geo& g, const Phys& p, const double* bW, const double* aW, const double* aT,
                   const double* alpha_new, const double* wp, const double* wn1, const double* Tn1, const double* rho,
                   const double* D, double* Tn1bar, double* wpbar, double* rhobar, double* Dbar) {
  ++g_launches, k_adj_species<<<lin_grid(g.N), TPB, 0, st>>>(g, p, bW, aW, aT, alpha_new, wp, wn1, Tn1, rho, D, Tn1bar,
                                                            wpbar, rhobar, Dbar);
}
void L_adj_energy(cudaStream_t st, const Geo& g, const Phys& p, const double* bT, const double* Tn, const double* Tn1,
                  const double* rho, const double* cp, const double* kc, double* Tnbar, double* rhobar, double* kbar,
                  double* cpbar, double* mdbar) {
  ++g_launches, k_adj_energy<<<lin_grid(g.N), TPB, 0, st>>>(g, p, bT, Tn, Tn1, rho, cp, kc, Tnbar, rhobar, kbar, cpbar,
                                                           mdbar);
}
void L_adj_source(cudaStream_t st, const Geo& g, const Phys& p, const double* aA, const double* alpha_n,
                  const double* alpha_new, const double* astar, const double* rgn, const double* mraw,
                  const double* scal, const double* rhobar, const double* kbar, const double* cpbar,
                  const double* Dbar, double jweight, double* aAn, double* rgbar, double* mdbar, double* mrbar,
                  double* part, double* acc_out) {
  int nb = red_grid(g.N);
  ++g_launches, k_adj_props_source<<<nb, TPB, 0, st>>>(g, p, aA, alpha_n, alpha_new, astar, rgn, mraw, scal, rhobar,
                                                      kbar, cpbar, Dbar, jweight, aAn, rgbar, mdbar, part);
  ++g_launches, k_adj_K<<<nb, TPB, 0, st>>>(g, p, part, nb, alpha_n, mraw, scal, mdbar, mrbar, aAn, acc_out);
}
void L_adj_K(cudaStream_t st, const Geo& g, const Phys& p, const double* part, int nblk, const double* alpha_n,
             const double* mraw, const double* scal, const double* mdbar, double* mrbar, double* aAn, double* acc_out) {
  ++g_launches, k_adj_K<<<nblk, TPB, 0, st>>>(g, p, part, nblk, alpha_n, mraw, scal, mdbar, mrbar, aAn, acc_out);
}
void L_adj_evap(cudaStream_t st, const Geo& g, const Phys& p, const double* alpha_n, const double* wp,
                const double* rgn, const int* adj, const double* mrbar, double* aAn, double* wpbar, double* rgbar,
                double* part, double* acc_out) {
  int nb = red_grid(g.N);
  ++g_launches, k_adj_evap<<<nb, TPB, 0, st>>>(g, p, alpha_n, wp, rgn, adj, mrbar, aAn, wpbar, rgbar, part);
  ++g_launches, k_adj_acc<<<1, TPB, 0, st>>>(part, nb, acc_out);
}
void L_adj_thermo(cudaStream_t st, const Geo& g, const Phys& p, const double* alpha_n, const double* Tn,
                  const double* wp, const double* rgn, const double* rgbar, const double* wpbar, double* Tnbar,
                  double* aW) {
  ++g_launches, k_adj_thermo<<<lin_grid(g.N), TPB, 0, st>>>(g, p, alpha_n, Tn, wp, rgn, rgbar, wpbar, Tnbar, aW);
}

}  // namespace dg
