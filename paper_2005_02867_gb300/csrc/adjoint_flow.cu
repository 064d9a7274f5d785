// Discrete adjoint of the step with flow: the evaporation flux with its convective part,
// the FCT advection of alpha (Eq. advection, with the limiter's branches held), energy and
// species with convection (Eqs. Teqn, speciesequation), the momentum predictor with
// buoyancy and the centripetal force (Eqs. NavierStokesModified, magneticfield), the
// Stefan source and the variable-density pressure equation (Eq. pequation) and the
// velocity correction.  The stage formulas below repeat the forward kernels' arithmetic
// over the tangent type of adjoint_ad.cuh; the linear systems are transposed by solving
// them again (every operator is symmetric), with the forward solution giving the
// derivative with respect to the operator's coefficients:
//   A x = b  =>  A mu = xbar,  bbar = mu,  (D_P)bar = -mu_P x_P,
//                (c_PQ)bar = -(mu_P - mu_Q)(x_P - x_Q)
// for the box operators y_P = D_P x_P + sum_Q c_PQ (x_P - x_Q).  FP64.
#include "adjoint_ad.cuh"
#include "kernels.h"

namespace dg {

__device__ __forceinline__ void scatter(const AdjT& T, int arr, long long idx, double gsum) {
  if (gsum == 0.0 || arr < 0) return;
  if (arr >= J_PAR_TAMB) atomicAdd(T.acc + (arr == J_PAR_TAMB ? AC_TAMB_BC : AC_DGAS), gsum);
  else atomicAdd(T.lam[arr] + idx, gsum);
}

// ---------------------------------------------------------------- ghost reads
// Cell field value with at most one index outside the domain, the forward kernels'
// cellg rules; amb_par: the fixed boundary value is the ambient temperature (a parameter)
__device__ Tan cellg_t(const Geo& g, Rd& rd, const double* f, int arr, int i, int j, int k, int rule, int amb_par,
                       double ambv, const double* const* U) {
  int a, side;
  if (i < 0) { a = 0; side = 0; i = 0; }
  else if (i >= g.n[0]) { a = 0; side = 1; i = g.n[0] - 1; }
  else if (j < 0) { a = 1; side = 0; j = 0; }
  else if (j >= g.n[1]) { a = 1; side = 1; j = g.n[1] - 1; }
  else if (k < 0) { a = 2; side = 0; k = 0; }
  else if (k >= g.n[2]) { a = 2; side = 1; k = g.n[2] - 1; }
  else return rd(f, arr, cidx(g, i, j, k));
  const int kind = bc_of(g, a, side);
  if (rule == R_ALPHA) return kind == BC_AXIS ? rd(f, arr, cidx(g, i, j, k)) : tc(0.0);
  if (rule == R_ZG || kind == BC_AXIS || kind == BC_WALL) return rd(f, arr, cidx(g, i, j, k));
  bool fixed = true;
  if (kind == BC_OPEN) {
    int fi = i, fj = j, fk = k;
    if (side) {
      if (a == 0) fi = g.n[0];
      else if (a == 1) fj = g.n[1];
      else fk = g.n[2];
    }
    const double un = U[a][fidx(g, a, fi, fj, fk)];
    fixed = (side ? un : -un) < 0.0;
  }
  const Tan vb = rd(f, arr, cidx(g, i, j, k));
  if (!fixed) return vb;
  const Tan am = amb_par ? rd.par(ambv, J_PAR_TAMB) : tc(ambv);
  return 2.0 * am - vb;
}

// face velocity of direction c with at most one index outside its array (the forward ufg)
__device__ Tan ufg_t(const Geo& g, Rd& rd, const double* uc, int arr, int c, int i, int j, int k) {
  const int m0 = g.n[0] + (c == 0), m1 = g.n[1] + (c == 1), m2 = g.n[2] + (c == 2);
  int a, q, m;
  if (i < 0 || i >= m0) { a = 0; q = i; m = m0; }
  else if (j < 0 || j >= m1) { a = 1; q = j; m = m1; }
  else if (k < 0 || k >= m2) { a = 2; q = k; m = m2; }
  else return rd(uc, arr, fidx(g, c, i, j, k));
  const int side = q < 0 ? 0 : 1;
  const int kind = bc_of(g, a, side);
  const int kk = side ? q - (m - 1) : -q;
  if (a == c) {
    const int qe = side ? m - 1 : 0;
    const Tan ub = rd(uc, arr, fidx(g, c, a == 0 ? qe : i, a == 1 ? qe : j, a == 2 ? qe : k));
    if (kind == BC_OPEN) return ub;
    const int qb = side ? m - 1 - kk : kk;
    const Tan v = rd(uc, arr, fidx(g, c, a == 0 ? qb : i, a == 1 ? qb : j, a == 2 ? qb : k));
    return 2.0 * ub - v;
  }
  const int qb = kind == BC_OPEN ? (side ? m - 1 : 0) : (side ? m - kk : kk - 1);
  const Tan v = rd(uc, arr, fidx(g, c, a == 0 ? qb : i, a == 1 ? qb : j, a == 2 ? qb : k));
  return (kind == BC_OPEN || kind == BC_AXIS) ? v : -v;
}

__device__ __forceinline__ Tan cellc_t(const Geo& g, Rd& rd, const double* f, int arr, int i, int j, int k) {
  i = i < 0 ? 0 : (i >= g.n[0] ? g.n[0] - 1 : i);
  j = j < 0 ? 0 : (j >= g.n[1] ? g.n[1] - 1 : j);
  k = k < 0 ? 0 : (k >= g.n[2] ? g.n[2] - 1 : k);
  return rd(f, arr, cidx(g, i, j, k));
}

// ---------------------------------------------------------------- S1: m_raw of an interface cell
// m_raw_P = -j_Q . grad(alpha)_P, j_Q = -rho_Q D_Q grad(omega')_Q + rho_Q omega'_Q v_Q at the
// adjacent gas cell Q (the forward step's choice)
template <int NA>
__device__ Tan f_mraw(const Geo& g, const Phys& p, const FlowIn& in, Rd& rd, long long id, long long qid) {
  int i, j, k, qi, qj, qk;
  decomp(id, g.n[0], g.n[1], i, j, k);
  decomp(qid, g.n[0], g.n[1], qi, qj, qk);
  Tan gr[3], gw[3], vc[3];
  const double* const* U = in.u;
  #pragma unroll
  for (int a = 0; a < NA; ++a) {
    int pp[3] = {i, j, k}, pm[3] = {i, j, k}, qp[3] = {qi, qj, qk}, qm[3] = {qi, qj, qk};
    pp[a] += 1; pm[a] -= 1; qp[a] += 1; qm[a] -= 1;
    gr[a] = (cellg_t(g, rd, in.alpha_n, J_ALPHA_N, pp[0], pp[1], pp[2], R_ALPHA, 0, 0.0, U) -
             cellg_t(g, rd, in.alpha_n, J_ALPHA_N, pm[0], pm[1], pm[2], R_ALPHA, 0, 0.0, U)) * (0.5 * g.ih[a]);
    gw[a] = (cellg_t(g, rd, in.wp, J_WP, qp[0], qp[1], qp[2], R_TO, 0, 0.0, U) -
             cellg_t(g, rd, in.wp, J_WP, qm[0], qm[1], qm[2], R_TO, 0, 0.0, U)) * (0.5 * g.ih[a]);
    int hq[3] = {qi, qj, qk};
    hq[a] += 1;
    vc[a] = 0.5 * (rd(U[a], J_U0 + a, fidx(g, a, qi, qj, qk)) + rd(U[a], J_U0 + a, fidx(g, a, hq[0], hq[1], hq[2])));
  }
  const Tan aQ = rd(in.alpha_n, J_ALPHA_N, qid), rgQ = rd(in.rgo, J_RGO, qid), wQ = rd(in.wp, J_WP, qid);
  const Tan rhoQ = aQ * p.rho_l + (1.0 - aQ) * rgQ;
  const Tan DQ = aQ * p.D_l + (1.0 - aQ) * rd.par(p.D_gas, J_PAR_DGAS);
  Tan s = tc(0.0);
  #pragma unroll
  for (int a = 0; a < NA; ++a) s = s + (-(rhoQ * DQ) * gw[a] + rhoQ * wQ * vc[a]) * gr[a];
  return -s;
}

// ---------------------------------------------------------------- S3: FCT advection
// face of direction A: low-order flux FL and antidiffusive flux AF
template <int A, int NA>
__device__ void f_adv_face(const Geo& g, const Phys& p, const FlowIn& in, Rd& rd, long long id, Tan& FL, Tan& AF) {
  constexpr int a = A;
  const int m0 = g.n[0] + (a == 0), m1 = g.n[1] + (a == 1);
  int f[3];
  decomp(id, m0, m1, f[0], f[1], f[2]);
  int L[3] = {f[0], f[1], f[2]}, R[3] = {f[0], f[1], f[2]};
  L[a] -= 1;
  const double* const* U = in.u;
  const Tan phi = rd(in.u[a], J_U0 + a, id) * (faceA(g, a, f[0]) * dt_of(p));
  const Tan aL = cellg_t(g, rd, in.astar, J_ASTAR, L[0], L[1], L[2], R_ALPHA, 0, 0.0, U);
  const Tan aR = cellg_t(g, rd, in.astar, J_ASTAR, R[0], R[1], R[2], R_ALPHA, 0, 0.0, U);
  const bool pos = phi.v >= 0.0;
  FL = phi * (pos ? aL : aR);
  AF = tc(0.0);
  if (f[a] > 0 && f[a] < g.n[a]) {
    int LL[3] = {L[0], L[1], L[2]}, RR[3] = {R[0], R[1], R[2]};
    LL[a] -= 1;
    RR[a] += 1;
    const Tan aLL = cellg_t(g, rd, in.astar, J_ASTAR, LL[0], LL[1], LL[2], R_ALPHA, 0, 0.0, U);
    const Tan aRR = cellg_t(g, rd, in.astar, J_ASTAR, RR[0], RR[1], RR[2], R_ALPHA, 0, 0.0, U);
    const Tan aVL = pos ? tvan_leer(aLL, aL, aR) : tvan_leer(aRR, aR, aL);
    Tan gf[3];
    #pragma unroll
    for (int b = 0; b < NA; ++b) {
      int Lp[3] = {L[0], L[1], L[2]}, Lm[3] = {L[0], L[1], L[2]}, Rp[3] = {R[0], R[1], R[2]}, Rm[3] = {R[0], R[1], R[2]};
      Lp[b] += 1; Lm[b] -= 1; Rp[b] += 1; Rm[b] -= 1;
      const Tan gLb = (cellg_t(g, rd, in.astar, J_ASTAR, Lp[0], Lp[1], Lp[2], R_ALPHA, 0, 0.0, U) -
                       cellg_t(g, rd, in.astar, J_ASTAR, Lm[0], Lm[1], Lm[2], R_ALPHA, 0, 0.0, U)) * (0.5 * g.ih[b]);
      const Tan gRb = (cellg_t(g, rd, in.astar, J_ASTAR, Rp[0], Rp[1], Rp[2], R_ALPHA, 0, 0.0, U) -
                       cellg_t(g, rd, in.astar, J_ASTAR, Rm[0], Rm[1], Rm[2], R_ALPHA, 0, 0.0, U)) * (0.5 * g.ih[b]);
      gf[b] = gLb + gRb;
    }
    Tan s2 = gf[0] * gf[0] + gf[1] * gf[1];
    if (NA == 3) s2 = s2 + gf[2] * gf[2];
    const Tan gfm = tsqrt(s2);
    const Tan ne = gfm.v > g.gthr ? gf[a] / gfm : tc(0.0);
    const Tan ac = 0.5 * (aL + aR);
    const Tan FH = phi * aVL + p.C_alpha * tabs(phi) * ne * ac * (1.0 - ac);
    AF = FH - FL;
  }
}

// alpha^L_P = alpha*_P - (net low-order flux) / V
template <int NA>
__device__ Tan f_adv_low(const Geo& g, const FlowIn& in, Rd& rd, long long id, int i, int j, int k) {
  Tan s = tc(0.0);
  #pragma unroll
  for (int a = 0; a < NA; ++a) {
    int hi[3] = {i, j, k};
    hi[a] += 1;
    s = s + (rd(in.FL[a], J_FL0 + a, fidx(g, a, hi[0], hi[1], hi[2])) - rd(in.FL[a], J_FL0 + a, fidx(g, a, i, j, k)));
  }
  return rd(in.astar, J_ASTAR, id) - s * (1.0 / cellV(g, i));
}

// Zalesak ratios R+ and R- of cell P
template <int NA>
__device__ void f_adv_limit(const Geo& g, const FlowIn& in, Rd& rd, long long id, int i, int j, int k, Tan& Rp,
                            Tan& Rm) {
  const Tan sP = rd(in.astar, J_ASTAR, id), lP = rd(in.aL, J_AL, id);
  Tan amax = tmax(sP, lP), amin = tmin(sP, lP);
  #pragma unroll
  for (int a = 0; a < NA; ++a)
    #pragma unroll
    for (int sh = -1; sh <= 1; sh += 2) {
      int q[3] = {i, j, k};
      q[a] += sh;
      if (q[a] < 0 || q[a] >= g.n[a]) continue;
      const long long qi = cidx(g, q[0], q[1], q[2]);
      const Tan sq = rd(in.astar, J_ASTAR, qi), lq = rd(in.aL, J_AL, qi);
      amax = tmax(amax, tmax(sq, lq));
      amin = tmin(amin, tmin(sq, lq));
    }
  amax = tmin(amax, tc(1.0));
  amin = tmax(amin, tc(0.0));
  Tan Pp = tc(0.0), Pm = tc(0.0);
  #pragma unroll
  for (int a = 0; a < NA; ++a) {
    int hi[3] = {i, j, k};
    hi[a] += 1;
    const Tan Alo = rd(in.AF[a], J_AF0 + a, fidx(g, a, i, j, k));
    const Tan Ahi = rd(in.AF[a], J_AF0 + a, fidx(g, a, hi[0], hi[1], hi[2]));
    Pp = Pp + tmax(tc(0.0), Alo) + tmax(tc(0.0), -Ahi);
    Pm = Pm + tmax(tc(0.0), -Alo) + tmax(tc(0.0), Ahi);
  }
  const double V = cellV(g, i);
  const Tan Qp = (amax - lP) * V, Qm = (lP - amin) * V;
  Rp = Pp.v > 0.0 && Qp.v > 0.0 ? tclamp01(Qp / Pp) : tc(0.0);
  Rm = Pm.v > 0.0 && Qm.v > 0.0 ? tclamp01(Qm / Pm) : tc(0.0);
}

// limited antidiffusive flux C A of the face (f0, f1, f2) of direction a
__device__ __forceinline__ Tan f_limited(const Geo& g, const FlowIn& in, Rd& rd, int a, int f0, int f1, int f2) {
  if (f0 < 0 || (a == 0 && (f0 == 0 || f0 == g.n[0])) || (a == 1 && (f1 == 0 || f1 == g.n[1])) ||
      (a == 2 && (f2 == 0 || f2 == g.n[2])))
    return tc(0.0);   // boundary faces carry no antidiffusive flux
  const Tan Af = rd(in.AF[a], J_AF0 + a, fidx(g, a, f0, f1, f2));
  int L[3] = {f0, f1, f2};
  L[a] -= 1;
  const long long li = cidx(g, L[0], L[1], L[2]), ri = cidx(g, f0, f1, f2);
  const Tan C = Af.v >= 0.0 ? tmin(rd(in.Rp, J_RP, ri), rd(in.Rm, J_RM, li))
                            : tmin(rd(in.Rp, J_RP, li), rd(in.Rm, J_RM, ri));
  return C * Af;
}

// alpha^{n+1} before clipping
template <int NA>
__device__ Tan f_adv_update(const Geo& g, const FlowIn& in, Rd& rd, long long id, int i, int j, int k) {
  Tan s = tc(0.0);
  #pragma unroll
  for (int a = 0; a < NA; ++a) {
    int hi[3] = {i, j, k};
    hi[a] += 1;
    s = s + (f_limited(g, in, rd, a, hi[0], hi[1], hi[2]) - f_limited(g, in, rd, a, i, j, k));
  }
  return rd(in.aL, J_AL, id) - s * (1.0 / cellV(g, i));
}

// ---------------------------------------------------------------- S5 / S6: scalar systems
// One row of the energy (mode 0) or species (mode 1) system: D_P, rhs_P and the couplings
// C_a[P] with the lower neighbours
template <int NA>
__device__ void f_scalar(const Geo& g, const Phys& p, int mode, const FlowIn& in, Rd& rd, long long id, Tan& Dout,
                         Tan& Rout, Tan Cout[3]) {
  int i, j, k;
  decomp(id, g.n[0], g.n[1], i, j, k);
  const double* const* U = in.u;
  const double* phi = mode == 0 ? in.T_n : in.wp;
  const int aphi = mode == 0 ? J_T_N : J_WP;
  const double V = cellV(g, i), idt = idt_of(p);
  auto gam = [&](long long q) -> Tan {
    return mode == 0 ? rd(in.kc, J_KC, q) : rd(in.rho, J_RHO, q) * rd(in.Dm, J_DM, q);
  };
  const Tan coef = mode == 0 ? rd(in.rho, J_RHO, id) * rd(in.cp, J_CP, id) : rd(in.rho, J_RHO, id);
  Tan dP = coef * V * idt;
  Tan r = coef * V * rd(phi, aphi, id) * idt;
  if (mode == 0) r = r + (-rd(in.mdot, J_MDOT, id) * p.Lv) * V;
  Tan net = tc(0.0), Fsum = tc(0.0);
  const Tan gP = gam(id);
  const bool pin = (mode == 1) && ige64(in.alpha1[id], 0.5);
  const int ci[3] = {i, j, k};
  #pragma unroll
  for (int a = 0; a < NA; ++a) {
    #pragma unroll
    for (int side = 0; side < 2; ++side) {
      int f[3] = {i, j, k};
      if (side) f[a] += 1;
      const Tan F = rd(U[a], J_U0 + a, fidx(g, a, f[0], f[1], f[2])) * faceA(g, a, f[0]);
      Tan val;
      if (f[a] == 0 || f[a] == g.n[a]) {
        const int kind = side ? g.bc[a][1] : g.bc[a][0];
        const bool inflow = side == 0 ? (F.v > 0.0) : (F.v < 0.0);
        if ((kind == BC_OPEN || kind == BC_FORCED) && inflow) val = mode == 0 ? rd.par(p.T_amb, J_PAR_TAMB) : tc(0.0);
        else val = rd(phi, aphi, id);
      } else {
        int L[3] = {f[0], f[1], f[2]};
        L[a] -= 1;
        int LL[3] = {L[0], L[1], L[2]}, RR[3] = {f[0], f[1], f[2]};
        LL[a] -= 1;
        RR[a] += 1;
        const Tan vL = rd(phi, aphi, cidx(g, L[0], L[1], L[2])), vR = rd(phi, aphi, cidx(g, f[0], f[1], f[2]));
        const double ambv = mode == 0 ? p.T_amb : 0.0;
        if (F.v >= 0.0) val = tlim_up(cellg_t(g, rd, phi, aphi, LL[0], LL[1], LL[2], R_TO, mode == 0, ambv, U), vL, vR);
        else val = tlim_up(cellg_t(g, rd, phi, aphi, RR[0], RR[1], RR[2], R_TO, mode == 0, ambv, U), vR, vL);
      }
      const double sgn = side ? 1.0 : -1.0;
      net = net + sgn * (F * val);
      Fsum = Fsum + sgn * F;
    }
    Tan cl = tc(0.0);
    if (ci[a] > 0) {
      int Lc[3] = {i, j, k};
      Lc[a] -= 1;
      const long long li = cidx(g, Lc[0], Lc[1], Lc[2]);
      const Tan gL = gam(li);
      cl = (2.0 * gL * gP / (gL + gP)) * (faceA(g, a, i) * g.ih[a]);
      if (mode == 1) {
        const bool lp = ige64(in.alpha1[li], 0.5);
        if (!pin && lp) { r = r + cl * rd(in.yq, J_YQ, li); dP = dP + cl; }
        if (pin || lp) cl = tc(0.0);
      }
    }
    Cout[a] = cl;
    if (mode == 1 && ci[a] < g.n[a] - 1 && !pin) {
      int Hc[3] = {i, j, k};
      Hc[a] += 1;
      const long long hi = cidx(g, Hc[0], Hc[1], Hc[2]);
      if (ige64(in.alpha1[hi], 0.5)) {
        const Tan gH = gam(hi);
        const Tan ch = (2.0 * gP * gH / (gP + gH)) * (faceA(g, a, Hc[0]) * g.ih[a]);
        r = r + ch * rd(in.yq, J_YQ, hi);
        dP = dP + ch;
      }
    }
    #pragma unroll
    for (int side = 0; side < 2; ++side) {
      const bool atb = side ? (ci[a] == g.n[a] - 1) : (ci[a] == 0);
      if (!atb) continue;
      const int kind = side ? g.bc[a][1] : g.bc[a][0];
      bool isdir = false;
      int f[3] = {i, j, k};
      if (side) f[a] += 1;
      if (kind == BC_FORCED) isdir = true;
      else if (kind == BC_OPEN) {
        const double un = U[a][fidx(g, a, f[0], f[1], f[2])];
        isdir = (side ? un : -un) < 0.0;
      }
      if (isdir) {
        const Tan cb = gP * (faceA(g, a, f[0]) * (2.0 * g.ih[a]));
        dP = dP + cb;
        r = r + cb * (mode == 0 ? rd.par(p.T_amb, J_PAR_TAMB) : tc(0.0));
      }
    }
  }
  r = r - coef * (net - rd(phi, aphi, id) * Fsum);
  if (pin) {
    const Tan dd = coef * V * idt;
    r = dd * rd(in.yq, J_YQ, id);
    dP = dd;
  }
  Dout = dP;
  Rout = r;
}

// ---------------------------------------------------------------- S7: momentum rows
template <int C, int NA>
__device__ void f_mom(const Geo& g, const Phys& p, const FlowIn& in, Rd& rd, long long id, Tan& Dout, Tan& Rout,
                      Tan Cout[3]) {
  constexpr int c = C;
  int m[3] = {g.n[0], g.n[1], g.n[2]};
  m[c] -= 1;
  int b[3];
  decomp(id, m[0], m[1], b[0], b[1], b[2]);
  int f[3] = {b[0], b[1], b[2]};
  f[c] += 1;
  int L[3] = {f[0], f[1], f[2]}, R[3] = {f[0], f[1], f[2]};
  L[c] -= 1;
  const double* const* U = in.u;
  const double* uc = U[c];
  const long long li = cidx(g, L[0], L[1], L[2]), ri = cidx(g, R[0], R[1], R[2]);
  const Tan rhoL = rd(in.rho, J_RHO, li), rhoR = rd(in.rho, J_RHO, ri);
  const Tan muL = rd(in.mu, J_MU, li), muR = rd(in.mu, J_MU, ri);
  const Tan rho_f = 0.5 * (rhoL + rhoR), mu_f = 0.5 * (muL + muR);
  double r_f = 0.0, V_f;
  if (g.axisym) {
    r_f = (c == 0) ? f[0] * g.h[0] : (f[0] + 0.5) * g.h[0];
    V_f = r_f * g.h[0] * g.h[1];
  } else {
    V_f = g.vol3;
  }
  const double A_f = V_f * g.ih[c];
  const Tan u_f = rd(uc, J_U0 + c, fidx(g, c, f[0], f[1], f[2]));
  const Tan rV = rho_f * V_f, muLR = muL + muR;
  Tan d = rV * idt_of(p);
  Tan r = d * u_f;
  Tan s_adv = tc(0.0), t_vT = tc(0.0), d_visc = tc(0.0);
  #pragma unroll
  for (int a = 0; a < NA; ++a) {
    Tan ubar;
    if (a == c) ubar = u_f;
    else {
      int La[3] = {L[0], L[1], L[2]}, Ra[3] = {R[0], R[1], R[2]};
      La[a] += 1;
      Ra[a] += 1;
      ubar = 0.25 * (((rd(U[a], J_U0 + a, fidx(g, a, L[0], L[1], L[2])) +
                       rd(U[a], J_U0 + a, fidx(g, a, La[0], La[1], La[2]))) +
                      rd(U[a], J_U0 + a, fidx(g, a, R[0], R[1], R[2]))) +
                     rd(U[a], J_U0 + a, fidx(g, a, Ra[0], Ra[1], Ra[2])));
    }
    Tan us[5];
    #pragma unroll
    for (int s = -2; s <= 2; ++s) {
      int q[3] = {f[0], f[1], f[2]};
      q[a] += s;
      us[s + 2] = ufg_t(g, rd, uc, J_U0 + c, c, q[0], q[1], q[2]);
    }
    Tan uplus, uminus;
    if (ubar.v >= 0.0) { uplus = tlim_up(us[1], us[2], us[3]); uminus = tlim_up(us[0], us[1], us[2]); }
    else { uplus = tlim_up(us[4], us[3], us[2]); uminus = tlim_up(us[3], us[2], us[1]); }
    s_adv = s_adv + ubar * (uplus - uminus) * g.ih[a];
    if (a == c) {
      double ApL, ApR;
      if (g.axisym && c == 0) { ApL = areaN(g, 0, (L[0] + 0.5) * g.h[0]); ApR = areaN(g, 0, (R[0] + 0.5) * g.h[0]); }
      else if (g.axisym) { ApL = ApR = areaN(g, 1, r_f); }
      else { ApL = ApR = areaN(g, c, 0.0); }
      const Tan kR = muR * (ApR * g.ih[c]), kL = muL * (ApL * g.ih[c]);
      t_vT = t_vT + (kR * (us[3] - us[2]) - kL * (us[2] - us[1]));
      Cout[c] = (b[c] > 0) ? kL : tc(0.0);
      if (b[c] == 0 && g.bc[c][0] != BC_OPEN) {
        int fb[3] = {f[0], f[1], f[2]};
        fb[c] = 0;
        d_visc = d_visc + kL;
        r = r + kL * rd(uc, J_U0 + c, fidx(g, c, fb[0], fb[1], fb[2]));
      }
      if (b[c] == m[c] - 1 && g.bc[c][1] != BC_OPEN) {
        int fb[3] = {f[0], f[1], f[2]};
        fb[c] = g.n[c];
        d_visc = d_visc + kR;
        r = r + kR * rd(uc, J_U0 + c, fidx(g, c, fb[0], fb[1], fb[2]));
      }
    } else {
      double App, Apm;
      if (g.axisym && a == 0) { App = areaN(g, 0, (f[0] + 1) * g.h[0]); Apm = areaN(g, 0, f[0] * g.h[0]); }
      else if (g.axisym) { App = Apm = areaN(g, 1, r_f); }
      else { App = Apm = areaN(g, a, 0.0); }
      int Lp[3] = {L[0], L[1], L[2]}, Rp[3] = {R[0], R[1], R[2]}, Lm[3] = {L[0], L[1], L[2]}, Rm[3] = {R[0], R[1], R[2]};
      Lp[a] += 1; Rp[a] += 1; Lm[a] -= 1; Rm[a] -= 1;
      const Tan mup = 0.25 * (muLR + cellc_t(g, rd, in.mu, J_MU, Lp[0], Lp[1], Lp[2]) +
                              cellc_t(g, rd, in.mu, J_MU, Rp[0], Rp[1], Rp[2]));
      const Tan mum = 0.25 * (muLR + cellc_t(g, rd, in.mu, J_MU, Lm[0], Lm[1], Lm[2]) +
                              cellc_t(g, rd, in.mu, J_MU, Rm[0], Rm[1], Rm[2]));
      const Tan kp = mup * (App * g.ih[a]), km = mum * (Apm * g.ih[a]);
      int La[3] = {L[0], L[1], L[2]}, Ra[3] = {R[0], R[1], R[2]};
      La[a] += 1;
      Ra[a] += 1;
      const Tan uaR_hi = rd(U[a], J_U0 + a, fidx(g, a, Ra[0], Ra[1], Ra[2]));
      const Tan uaL_hi = rd(U[a], J_U0 + a, fidx(g, a, La[0], La[1], La[2]));
      const Tan uaR_lo = rd(U[a], J_U0 + a, fidx(g, a, R[0], R[1], R[2]));
      const Tan uaL_lo = rd(U[a], J_U0 + a, fidx(g, a, L[0], L[1], L[2]));
      t_vT = t_vT + (mup * App * (uaR_hi - uaL_hi) - mum * Apm * (uaR_lo - uaL_lo)) * g.ih[c];
      Cout[a] = (b[a] > 0) ? km : tc(0.0);
      if (b[a] == 0 && (g.bc[a][0] == BC_WALL || g.bc[a][0] == BC_FORCED)) d_visc = d_visc + 2.0 * km;
      if (b[a] == m[a] - 1 && (g.bc[a][1] == BC_WALL || g.bc[a][1] == BC_FORCED)) d_visc = d_visc + 2.0 * kp;
    }
  }
  if (g.axisym && c == 0 && r_f > 0.0) d_visc = d_visc + 2.0 * mu_f * V_f / (r_f * r_f);
  double gx = 0.0;
  #pragma unroll
  for (int a = 0; a < NA; ++a) {
    const double xa = (a == c) ? f[a] * g.h[a] : (f[a] + 0.5) * g.h[a];
    gx = gx + p.g[a] * xa;
  }
  const double xiL = in.xi[li], xiR = in.xi[ri];
  const Tan raL = rhoL * rd(in.alpha1, J_ALPHA1, li), raR = rhoR * rd(in.alpha1, J_ALPHA1, ri);
  const Tan t_force = A_f * ((0.5 * (raL + raR) * (xiR - xiL) - gx * (rhoR - rhoL)) -
                             (rd(in.p_n, J_P_N, ri) - rd(in.p_n, J_P_N, li)));
  Dout = d + d_visc;
  Rout = r - rV * s_adv + t_vT + t_force;
}

// ---------------------------------------------------------------- S8: pressure rows
template <int NA>
__device__ void f_poisson(const Geo& g, const Phys& p, const FlowIn& in, Rd& rd, long long id, Tan& Dout, Tan& Rout,
                          Tan Cout[3]) {
  int i, j, k;
  decomp(id, g.n[0], g.n[1], i, j, k);
  const double* const* U = in.u;
  const int ci[3] = {i, j, k};
  Tan adv = tc(0.0);
  #pragma unroll
  for (int a = 0; a < NA; ++a) {
    int hi[3] = {i, j, k};
    hi[a] += 1;
    const Tan vc = 0.5 * (rd(U[a], J_U0 + a, fidx(g, a, i, j, k)) + rd(U[a], J_U0 + a, fidx(g, a, hi[0], hi[1], hi[2])));
    int qp[3] = {i, j, k}, qm[3] = {i, j, k};
    qp[a] += 1;
    qm[a] -= 1;
    const Tan gr = (cellg_t(g, rd, in.rgn, J_RGN, qp[0], qp[1], qp[2], R_ZG, 0, 0.0, U) -
                    cellg_t(g, rd, in.rgn, J_RGN, qm[0], qm[1], qm[2], R_ZG, 0, 0.0, U)) * (0.5 * g.ih[a]);
    adv = adv + vc * gr;
  }
  const Tan rn = rd(in.rgn, J_RGN, id);
  const Tan irn = 1.0 / rn;
  const Tan s = rd(in.mdot, J_MDOT, id) * (irn - p.irho_l) -
                (1.0 - rd(in.alpha1, J_ALPHA1, id)) * irn * ((rn - rd(in.rgo, J_RGO, id)) * idt_of(p) + adv);
  Tan dg = tc(0.0), div = tc(0.0);
  const Tan rP = rd(in.rho, J_RHO, id);
  #pragma unroll
  for (int a = 0; a < NA; ++a) {
    int hi[3] = {i, j, k};
    hi[a] += 1;
    div = div + (rd(in.us[a], J_US0 + a, fidx(g, a, hi[0], hi[1], hi[2])) * faceA(g, a, hi[0]) -
                 rd(in.us[a], J_US0 + a, fidx(g, a, i, j, k)) * faceA(g, a, i));
    Tan cl = tc(0.0);
    if (ci[a] > 0) {
      int Lc[3] = {i, j, k};
      Lc[a] -= 1;
      cl = (faceA(g, a, i) * g.ih[a]) * (2.0 / (rd(in.rho, J_RHO, cidx(g, Lc[0], Lc[1], Lc[2])) + rP));
    }
    Cout[a] = cl;
    if (ci[a] == 0 && g.bc[a][0] == BC_OPEN) dg = dg + (faceA(g, a, i) * (2.0 * g.ih[a])) / rP;
    if (ci[a] == g.n[a] - 1 && g.bc[a][1] == BC_OPEN) dg = dg + (faceA(g, a, hi[0]) * (2.0 * g.ih[a])) / rP;
  }
  Dout = dg;
  Rout = (s * cellV(g, i) - div) * idt_of(p);
}

// ---------------------------------------------------------------- S10: velocity correction
template <int C>
__device__ Tan f_correct(const Geo& g, const Phys& p, const FlowIn& in, Rd& rd, long long id) {
  constexpr int c = C;
  const int m0 = g.n[0] + (c == 0), m1 = g.n[1] + (c == 1);
  int f[3];
  decomp(id, m0, m1, f[0], f[1], f[2]);
  const double A = faceA(g, c, f[0]);
  Tan corr = tc(0.0);
  if (A > 0.0) {
    int L[3] = {f[0], f[1], f[2]};
    L[c] -= 1;
    if (f[c] > 0 && f[c] < g.n[c]) {
      const long long li = cidx(g, L[0], L[1], L[2]), ri = cidx(g, f[0], f[1], f[2]);
      corr = (dt_of(p) * g.ih[c]) * (2.0 / (rd(in.rho, J_RHO, li) + rd(in.rho, J_RHO, ri))) *
             (rd(in.dp, J_DP, ri) - rd(in.dp, J_DP, li));
    } else {
      const int side = f[c] == 0 ? 0 : 1;
      if ((side ? g.bc[c][1] : g.bc[c][0]) == BC_OPEN) {
        const long long pi = side ? cidx(g, L[0], L[1], L[2]) : cidx(g, f[0], f[1], f[2]);
        const Tan bA = (2.0 * g.ih[c]) / rd(in.rho, J_RHO, pi);
        const Tan dpp = rd(in.dp, J_DP, pi);
        corr = side ? dt_of(p) * bA * (0.0 - dpp) : dt_of(p) * bA * dpp;
      }
    }
  }
  return rd(in.us[c], J_US0 + c, id) - corr;
}

// ================================================================ adjoint kernels
// Each thread owns one output row (a face or a cell): it forms the weights of its outputs,
// evaluates the formula once to count its reads, then once per read with that read seeded,
// and adds the weighted derivative into the read's adjoint.
#define ADJ_EACH_READ(EVAL, GSUM)                  \
  {                                                \
    Rd r0(-1);                                     \
    EVAL(r0);                                      \
    const int nr = r0.cnt;                         \
    for (int s_ = 0; s_ < nr; ++s_) {              \
      Rd rd(s_);                                   \
      EVAL(rd);                                    \
      scatter(T, rd.arr, rd.idx, (GSUM));          \
    }                                              \
  }

template <int C>
__global__ void k_adjf_correct(Geo g, Phys p, FlowIn in, AdjT T, const double* lU) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= nfaces(g, C)) return;
  const double w = lU[id];
  if (w == 0.0) return;
  Tan u;
  auto eval = [&](Rd& rd) { u = f_correct<C>(g, p, in, rd, id); };
  ADJ_EACH_READ(eval, w * u.t)
}

// weights of a box row: rhs mu_P, diagonal -mu_P x_P, coupling with the lower neighbour
// along a -(mu_P - mu_Q)(x_P - x_Q)
__device__ __forceinline__ void box_weights(const int m[3], int na, long long id, const int b[3], const double* mu,
                                            const double* x, double& wr, double& wD, double wc[3]) {
  wr = mu[id];
  wD = -mu[id] * x[id];
  const long long st[3] = {1, (long long)m[0], (long long)m[0] * m[1]};
  for (int a = 0; a < 3; ++a) {
    wc[a] = 0.0;
    if (a < na && b[a] > 0) wc[a] = -(mu[id] - mu[id - st[a]]) * (x[id] - x[id - st[a]]);
  }
}

template <int NA>
__global__ void k_adjf_poisson(Geo g, Phys p, FlowIn in, AdjT T, const double* mu, const double* x) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  int b[3];
  decomp(id, g.n[0], g.n[1], b[0], b[1], b[2]);
  double wr, wD, wc[3];
  box_weights(g.n, NA, id, b, mu, x, wr, wD, wc);
  Tan D, R, Cc[3];
  auto eval = [&](Rd& rd) { f_poisson<NA>(g, p, in, rd, id, D, R, Cc); };
  ADJ_EACH_READ(eval, wr * R.t + wD * D.t + wc[0] * Cc[0].t + wc[1] * Cc[1].t + (NA == 3 ? wc[2] * Cc[2].t : 0.0))
}

template <int C, int NA>
__global__ void k_adjf_mom(Geo g, Phys p, FlowIn in, AdjT T, const double* mu, const double* x) {
  int m[3] = {g.n[0], g.n[1], g.n[2]};
  m[C] -= 1;
  const long long nb = (long long)m[0] * m[1] * m[2];
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= nb) return;
  int b[3];
  decomp(id, m[0], m[1], b[0], b[1], b[2]);
  double wr, wD, wc[3];
  box_weights(m, NA, id, b, mu, x, wr, wD, wc);
  Tan D, R, Cc[3] = {tc(0.0), tc(0.0), tc(0.0)};
  auto eval = [&](Rd& rd) { f_mom<C, NA>(g, p, in, rd, id, D, R, Cc); };
  ADJ_EACH_READ(eval, wr * R.t + wD * D.t + wc[0] * Cc[0].t + wc[1] * Cc[1].t + (NA == 3 ? wc[2] * Cc[2].t : 0.0))
}

template <int NA>
__global__ void k_adjf_scalar(Geo g, Phys p, FlowIn in, AdjT T, int mode, const double* mu, const double* x) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  int b[3];
  decomp(id, g.n[0], g.n[1], b[0], b[1], b[2]);
  double wr, wD, wc[3];
  box_weights(g.n, NA, id, b, mu, x, wr, wD, wc);
  Tan D, R, Cc[3];
  auto eval = [&](Rd& rd) { f_scalar<NA>(g, p, mode, in, rd, id, D, R, Cc); };
  ADJ_EACH_READ(eval, wr * R.t + wD * D.t + wc[0] * Cc[0].t + wc[1] * Cc[1].t + (NA == 3 ? wc[2] * Cc[2].t : 0.0))
}

// FCT, in reverse: the update (alpha^{n+1} before clipping; a clipped cell passes nothing),
// the limiter ratios, the low-order solution, the face fluxes
template <int NA>
__global__ void k_adjf_update(Geo g, Phys p, FlowIn in, AdjT T) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  const double w = T.lam[J_ALPHA1][id];
  if (w == 0.0) return;
  int i, j, k;
  decomp(id, g.n[0], g.n[1], i, j, k);
  Tan an;
  auto eval = [&](Rd& rd) { an = f_adv_update<NA>(g, in, rd, id, i, j, k); };
  {
    Rd r0(-1);
    eval(r0);
    if (iclamp01(an.v) != an.v) return;   // clipped: alpha^{n+1} is the bound
  }
  ADJ_EACH_READ(eval, w * an.t)
}

template <int NA>
__global__ void k_adjf_limit(Geo g, Phys p, FlowIn in, AdjT T) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  const double wp = T.lam[J_RP][id], wm = T.lam[J_RM][id];
  if (wp == 0.0 && wm == 0.0) return;
  int i, j, k;
  decomp(id, g.n[0], g.n[1], i, j, k);
  Tan Rp, Rm;
  auto eval = [&](Rd& rd) { f_adv_limit<NA>(g, in, rd, id, i, j, k, Rp, Rm); };
  ADJ_EACH_READ(eval, wp * Rp.t + wm * Rm.t)
}

template <int NA>
__global__ void k_adjf_low(Geo g, Phys p, FlowIn in, AdjT T) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  const double w = T.lam[J_AL][id];
  if (w == 0.0) return;
  int i, j, k;
  decomp(id, g.n[0], g.n[1], i, j, k);
  Tan aL;
  auto eval = [&](Rd& rd) { aL = f_adv_low<NA>(g, in, rd, id, i, j, k); };
  ADJ_EACH_READ(eval, w * aL.t)
}

template <int A, int NA>
__global__ void k_adjf_face(Geo g, Phys p, FlowIn in, AdjT T) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= nfaces(g, A)) return;
  const double wl = T.lam[J_FL0 + A][id], wa = T.lam[J_AF0 + A][id];
  if (wl == 0.0 && wa == 0.0) return;
  Tan FL, AF;
  auto eval = [&](Rd& rd) { f_adv_face<A, NA>(g, p, in, rd, id, FL, AF); };
  ADJ_EACH_READ(eval, wl * FL.t + wa * AF.t)
}

template <int NA>
__global__ void k_adjf_mraw(Geo g, Phys p, FlowIn in, AdjT T, const double* mrbar) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  const int q = in.adj[id];
  const double w = mrbar[id];
  if (q < 0 || w == 0.0) return;
  Tan m;
  auto eval = [&](Rd& rd) { m = f_mraw<NA>(g, p, in, rd, id, q); };
  ADJ_EACH_READ(eval, w * m.t)
}

// ---------------------------------------------------------------- pointwise stages
template <int C>
__global__ void k_adjf_box_gather(Geo g, const double* faces, double* box) {
  int m[3] = {g.n[0], g.n[1], g.n[2]};
  m[C] -= 1;
  const long long nb = (long long)m[0] * m[1] * m[2];
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= nb) return;
  int b[3];
  decomp(id, m[0], m[1], b[0], b[1], b[2]);
  b[C] += 1;
  box[id] = faces[fidx(g, C, b[0], b[1], b[2])];
}

// adjoint of u* (faces) into the box right-hand side: interior faces, plus the open boundary
// faces that copied their interior neighbour; other boundary faces kept u^n (into lun)
template <int C>
__global__ void k_adjf_box_rhs(Geo g, const double* lus, double* box, double* lun) {
  const long long nf = nfaces(g, C);
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= nf) return;
  const int m0 = g.n[0] + (C == 0), m1 = g.n[1] + (C == 1);
  int f[3];
  decomp(id, m0, m1, f[0], f[1], f[2]);
  int mb[3] = {g.n[0], g.n[1], g.n[2]};
  mb[C] -= 1;
  auto bidx = [&](int fc) {
    int b[3] = {f[0], f[1], f[2]};
    b[C] = fc - 1;
    return (long long)b[0] + (long long)mb[0] * ((long long)b[1] + (long long)mb[1] * b[2]);
  };
  const double w = lus[id];
  if (f[C] > 0 && f[C] < g.n[C]) { atomicAdd(box + bidx(f[C]), w); return; }
  const int side = f[C] == 0 ? 0 : 1;
  if ((side ? g.bc[C][1] : g.bc[C][0]) == BC_OPEN) atomicAdd(box + bidx(side ? g.n[C] - 1 : 1), w);
  else lun[id] += w;
}

// rho_G^{n+1} = P / (R T m(omega)), m = omega / M_l + (1 - omega) / M_g
__global__ void k_adjf_rhoG(Geo g, Phys p, const double* T1, const double* w1, const double* lrgn, double* lT1,
                            double* lW1) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  const double rb = lrgn[id];
  if (rb == 0.0) return;
  const double T = T1[id], w = w1[id];
  const double m = w * p.iM_l + (1.0 - w) * p.iM_g;
  const double R = rho_gas(p, T, w);
  lT1[id] += -rb * R / T;
  lW1[id] += -rb * R * (p.iM_l - p.iM_g) / m;
}

// pinned species rows take Y_eq(T^{n+1}) where alpha^{n+1} >= 1/2
__global__ void k_adjf_yq(Geo g, Phys p, const double* T1, const double* alpha1, const double* lyq, double* lT1) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  if (alpha1[id] < 0.5 || lyq[id] == 0.0) return;
  lT1[id] += lyq[id] * dYeq_dT(p, T1[id]);
}

// mixture properties at alpha^{n+1}, rho_G^n, omega' (S4)
__global__ void k_adjf_props(Geo g, Phys p, FlowIn in, AdjT T) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double dg = 0.0;
  if (id < g.N) {
    const double a1 = in.alpha1[id], rg = in.rgo[id], w = in.wp[id];
    const double lr = T.lam[J_RHO][id], lm = T.lam[J_MU][id], lk = T.lam[J_KC][id], lc = T.lam[J_CP][id],
                 ld = T.lam[J_DM][id];
    const double cpG = w * p.cp_v + (1.0 - w) * p.cp_g;
    T.lam[J_ALPHA1][id] += lr * (p.rho_l - rg) + lm * (p.mu_l - p.mu_g) + lk * (p.k_l - p.k_g) + lc * (p.cp_l - cpG) +
                           ld * (p.D_l - p.D_gas);
    T.lam[J_RGO][id] += lr * (1.0 - a1);
    T.lam[J_WP][id] += lc * (1.0 - a1) * (p.cp_v - p.cp_g);
    dg = ld * (1.0 - a1);
  }
  for (int o = 16; o > 0; o >>= 1) dg += __shfl_down_sync(0xffffffffu, dg, o);
  if ((threadIdx.x & 31) == 0 && dg != 0.0) atomicAdd(T.acc + AC_DGAS, dg);
}

// alpha* = alpha^n - dt mdot / rho_L where m_raw != 0 (mdot capped at rho_L alpha^n / dt), J =
// sum over the steps of jweight sum mdot V; the final adjoint of mdot (0 where capped) stays
// in lam[J_MDOT] and the block sums {0, mdbar f m_raw, m_raw V, f m_raw V} go to part
__global__ void k_adjf_source(Geo g, Phys p, FlowIn in, AdjT T, const double* mraw, const double* scal,
                              double jweight, double* part) {
  double acc[4] = {0, 0, 0, 0};
  const double K = scal[SC_K];
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < g.N; id += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    decomp(id, g.n[0], g.n[1], i, j, k);
    const double V = cellV(g, i);
    const double asb = T.lam[J_ASTAR][id];
    double md = T.lam[J_MDOT][id] + jweight * V;
    double aAn = asb;
    const double mr = mraw[id], an = in.alpha_n[id];
    const double f = sqrt(an * (1.0 - an));
    if (mr != 0.0) {
      md += -dt_of(p) * asb / p.rho_l;
      const double m_unc = (K == 0.0) ? 0.0 : K * f * mr;
      const double cap = p.rho_l * an * idt_of(p);
      if (m_unc > cap) {
        aAn += md * p.rho_l * idt_of(p);
        md = 0.0;
      }
    } else {
      md = 0.0;   // mdot = 0 there whatever the inputs
    }
    T.lam[J_MDOT][id] = md;
    T.lam[J_ALPHA_N][id] += aAn;
    acc[1] += md * f * mr;
    acc[2] += mr * V;
    acc[3] += f * mr * V;
  }
  block_sum_store<4>(acc, part);
}

// ---------------------------------------------------------------- launchers
void L_adjf_correct(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, const AdjT& T,
                    double* const lU[3]) {
  ++g_launches, k_adjf_correct<0><<<lin_grid(nfaces(g, 0)), TPB, 0, st>>>(g, p, in, T, lU[0]);
  ++g_launches, k_adjf_correct<1><<<lin_grid(nfaces(g, 1)), TPB, 0, st>>>(g, p, in, T, lU[1]);
  if (nact(g) == 3) ++g_launches, k_adjf_correct<2><<<lin_grid(nfaces(g, 2)), TPB, 0, st>>>(g, p, in, T, lU[2]);
}
void L_adjf_poisson(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, const AdjT& T, const double* mu,
                    const double* x) {
  ++g_launches;
  if (nact(g) == 3) k_adjf_poisson<3><<<lin_grid(g.N), TPB, 0, st>>>(g, p, in, T, mu, x);
  else k_adjf_poisson<2><<<lin_grid(g.N), TPB, 0, st>>>(g, p, in, T, mu, x);
}
void L_adjf_mom(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, const AdjT& T, int c,
                const double* mu, const double* x) {
  int m[3] = {g.n[0], g.n[1], g.n[2]};
  m[c] -= 1;
  const int gr = lin_grid((long long)m[0] * m[1] * m[2]);
  ++g_launches;
  if (nact(g) == 3) {
    if (c == 0) k_adjf_mom<0, 3><<<gr, TPB, 0, st>>>(g, p, in, T, mu, x);
    else if (c == 1) k_adjf_mom<1, 3><<<gr, TPB, 0, st>>>(g, p, in, T, mu, x);
    else k_adjf_mom<2, 3><<<gr, TPB, 0, st>>>(g, p, in, T, mu, x);
  } else {
    if (c == 0) k_adjf_mom<0, 2><<<gr, TPB, 0, st>>>(g, p, in, T, mu, x);
    else k_adjf_mom<1, 2><<<gr, TPB, 0, st>>>(g, p, in, T, mu, x);
  }
}
void L_adjf_scalar(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, const AdjT& T, int mode,
                   const double* mu, const double* x) {
  ++g_launches;
  if (nact(g) == 3) k_adjf_scalar<3><<<lin_grid(g.N), TPB, 0, st>>>(g, p, in, T, mode, mu, x);
  else k_adjf_scalar<2><<<lin_grid(g.N), TPB, 0, st>>>(g, p, in, T, mode, mu, x);
}
void L_adjf_fct(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, const AdjT& T) {
  const int gc = lin_grid(g.N);
  if (nact(g) == 3) {
    ++g_launches, k_adjf_update<3><<<gc, TPB, 0, st>>>(g, p, in, T);
    ++g_launches, k_adjf_limit<3><<<gc, TPB, 0, st>>>(g, p, in, T);
    ++g_launches, k_adjf_low<3><<<gc, TPB, 0, st>>>(g, p, in, T);
    ++g_launches, k_adjf_face<0, 3><<<lin_grid(nfaces(g, 0)), TPB, 0, st>>>(g, p, in, T);
    ++g_launches, k_adjf_face<1, 3><<<lin_grid(nfaces(g, 1)), TPB, 0, st>>>(g, p, in, T);
    ++g_launches, k_adjf_face<2, 3><<<lin_grid(nfaces(g, 2)), TPB, 0, st>>>(g, p, in, T);
  } else {
    ++g_launches, k_adjf_update<2><<<gc, TPB, 0, st>>>(g, p, in, T);
    ++g_launches, k_adjf_limit<2><<<gc, TPB, 0, st>>>(g, p, in, T);
    ++g_launches, k_adjf_low<2><<<gc, TPB, 0, st>>>(g, p, in, T);
    ++g_launches, k_adjf_face<0, 2><<<lin_grid(nfaces(g, 0)), TPB, 0, st>>>(g, p, in, T);
    ++g_launches, k_adjf_face<1, 2><<<lin_grid(nfaces(g, 1)), TPB, 0, st>>>(g, p, in, T);
  }
}
void L_adjf_mraw(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, const AdjT& T, const double* mrbar) {
  ++g_launches;
  if (nact(g) == 3) k_adjf_mraw<3><<<lin_grid(g.N), TPB, 0, st>>>(g, p, in, T, mrbar);
  else k_adjf_mraw<2><<<lin_grid(g.N), TPB, 0, st>>>(g, p, in, T, mrbar);
}
void L_adjf_box_gather(cudaStream_t st, const Geo& g, int c, const double* faces, double* box) {
  int m[3] = {g.n[0], g.n[1], g.n[2]};
  m[c] -= 1;
  const int gr = lin_grid((long long)m[0] * m[1] * m[2]);
  ++g_launches;
  if (c == 0) k_adjf_box_gather<0><<<gr, TPB, 0, st>>>(g, faces, box);
  else if (c == 1) k_adjf_box_gather<1><<<gr, TPB, 0, st>>>(g, faces, box);
  else k_adjf_box_gather<2><<<gr, TPB, 0, st>>>(g, faces, box);
}
void L_adjf_box_rhs(cudaStream_t st, const Geo& g, int c, const double* lus, double* box, double* lun) {
  const int gr = lin_grid(nfaces(g, c));
  ++g_launches;
  if (c == 0) k_adjf_box_rhs<0><<<gr, TPB, 0, st>>>(g, lus, box, lun);
  else if (c == 1) k_adjf_box_rhs<1><<<gr, TPB, 0, st>>>(g, lus, box, lun);
  else k_adjf_box_rhs<2><<<gr, TPB, 0, st>>>(g, lus, box, lun);
}
void L_adjf_rhoG(cudaStream_t st, const Geo& g, const Phys& p, const double* T1, const double* w1, const double* lrgn,
                 double* lT1, double* lW1) {
  ++g_launches, k_adjf_rhoG<<<lin_grid(g.N), TPB, 0, st>>>(g, p, T1, w1, lrgn, lT1, lW1);
}
void L_adjf_yq(cudaStream_t st, const Geo& g, const Phys& p, const double* T1, const double* alpha1,
               const double* lyq, double* lT1) {
  ++g_launches, k_adjf_yq<<<lin_grid(g.N), TPB, 0, st>>>(g, p, T1, alpha1, lyq, lT1);
}
void L_adjf_props(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, const AdjT& T) {
  ++g_launches, k_adjf_props<<<lin_grid(g.N), TPB, 0, st>>>(g, p, in, T);
}
void L_adjf_source(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, const AdjT& T,
                   const double* mraw, const double* scal, double jweight, double* mrbar, double* part) {
  const int nb = red_grid(g.N);
  ++g_launches, k_adjf_source<<<nb, TPB, 0, st>>>(g, p, in, T, mraw, scal, jweight, part);
  L_adj_K(st, g, p, part, nb, in.alpha_n, mraw, scal, T.lam[J_MDOT], mrbar, T.lam[J_ALPHA_N], T.acc);
}

// ================================================================ forward check of the formulas
// The stage formulas evaluated without a seed reproduce the forward kernels' values; these
// kernels record max |formula - forward| and max |forward| per check slot (non-negative
// binary64 compared as unsigned encodings)
__device__ __forceinline__ void chk_put(unsigned long long* chk, int slot, double diff, double ref) {
  atomicMax(chk + 2 * slot, (unsigned long long)__double_as_longlong(fabs(diff)));
  atomicMax(chk + 2 * slot + 1, (unsigned long long)__double_as_longlong(fabs(ref)));
}

template <int NA>
__global__ void k_chk_cells(Geo g, Phys p, FlowIn in, const double* mraw, unsigned long long* chk) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  int i, j, k;
  decomp(id, g.n[0], g.n[1], i, j, k);
  Rd rd(-1);
  const Tan aL = f_adv_low<NA>(g, in, rd, id, i, j, k);
  chk_put(chk, CHK_AL, aL.v - in.aL[id], in.aL[id]);
  Tan Rp, Rm;
  f_adv_limit<NA>(g, in, rd, id, i, j, k, Rp, Rm);
  chk_put(chk, CHK_RP, Rp.v - in.Rp[id], in.Rp[id]);
  chk_put(chk, CHK_RM, Rm.v - in.Rm[id], in.Rm[id]);
  const Tan an = f_adv_update<NA>(g, in, rd, id, i, j, k);
  chk_put(chk, CHK_ALPHA1, iclamp01(an.v) - in.alpha1[id], in.alpha1[id]);
  if (in.adj[id] >= 0) {
    const Tan m = f_mraw<NA>(g, p, in, rd, id, in.adj[id]);
    chk_put(chk, CHK_MRAW, m.v - mraw[id], mraw[id]);
  }
}

template <int A, int NA>
__global__ void k_chk_faces(Geo g, Phys p, FlowIn in, const double* unew, unsigned long long* chk) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= nfaces(g, A)) return;
  Rd rd(-1);
  Tan FL, AF;
  f_adv_face<A, NA>(g, p, in, rd, id, FL, AF);
  chk_put(chk, CHK_FL, FL.v - in.FL[A][id], in.FL[A][id]);
  chk_put(chk, CHK_AF, AF.v - in.AF[A][id], in.AF[A][id]);
  const Tan u = f_correct<A>(g, p, in, rd, id);
  chk_put(chk, CHK_CORRECT, u.v - unew[id], unew[id]);
}

// rows of an assembled box system (kind 0 energy, 1 species, 2 pressure, 3 + c momentum c)
template <int NA>
__global__ void k_chk_rows(Geo g, Phys p, FlowIn in, int kind, const double* D, const double* c0, const double* c1,
                           const double* c2, const double* rhs, unsigned long long* chk) {
  int m[3] = {g.n[0], g.n[1], g.n[2]};
  if (kind >= 3) m[kind - 3] -= 1;
  const long long nb = (long long)m[0] * m[1] * m[2];
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= nb) return;
  Rd rd(-1);
  Tan Dv, Rv, Cv[3] = {tc(0.0), tc(0.0), tc(0.0)};
  int slot;
  if (kind <= 1) { f_scalar<NA>(g, p, kind, in, rd, id, Dv, Rv, Cv); slot = kind == 0 ? CHK_ENERGY : CHK_SPECIES; }
  else if (kind == 2) { f_poisson<NA>(g, p, in, rd, id, Dv, Rv, Cv); slot = CHK_POISSON; }
  else {
    slot = CHK_MOM;
    if (kind == 3) f_mom<0, NA>(g, p, in, rd, id, Dv, Rv, Cv);
    else if (kind == 4) f_mom<1, NA>(g, p, in, rd, id, Dv, Rv, Cv);
    else if (NA == 3) f_mom<(NA == 3 ? 2 : 1), NA>(g, p, in, rd, id, Dv, Rv, Cv);
  }
  chk_put(chk, slot, Dv.v - D[id], D[id]);
  chk_put(chk, slot + 1, Rv.v - rhs[id], rhs[id]);
  const double* C[3] = {c0, c1, c2};
  for (int a = 0; a < NA; ++a) chk_put(chk, slot + 2, Cv[a].v - C[a][id], C[a][id]);
}

void L_chk_cells(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, const double* mraw,
                 unsigned long long* chk) {
  ++g_launches;
  if (nact(g) == 3) k_chk_cells<3><<<lin_grid(g.N), TPB, 0, st>>>(g, p, in, mraw, chk);
  else k_chk_cells<2><<<lin_grid(g.N), TPB, 0, st>>>(g, p, in, mraw, chk);
}
void L_chk_faces(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, double* const unew[3],
                 unsigned long long* chk) {
  if (nact(g) == 3) {
    ++g_launches, k_chk_faces<0, 3><<<lin_grid(nfaces(g, 0)), TPB, 0, st>>>(g, p, in, unew[0], chk);
    ++g_launches, k_chk_faces<1, 3><<<lin_grid(nfaces(g, 1)), TPB, 0, st>>>(g, p, in, unew[1], chk);
    ++g_launches, k_chk_faces<2, 3><<<lin_grid(nfaces(g, 2)), TPB, 0, st>>>(g, p, in, unew[2], chk);
  } else {
    ++g_launches, k_chk_faces<0, 2><<<lin_grid(nfaces(g, 0)), TPB, 0, st>>>(g, p, in, unew[0], chk);
    ++g_launches, k_chk_faces<1, 2><<<lin_grid(nfaces(g, 1)), TPB, 0, st>>>(g, p, in, unew[1], chk);
  }
}
void L_chk_rows(cudaStream_t st, const Geo& g, const Phys& p, const FlowIn& in, int kind, const double* D,
                double* const C[3], const double* rhs, unsigned long long* chk) {
  int m[3] = {g.n[0], g.n[1], g.n[2]};
  if (kind >= 3) m[kind - 3] -= 1;
  const int gr = lin_grid((long long)m[0] * m[1] * m[2]);
  const double* c2 = C[2] ? C[2] : C[0];
  ++g_launches;
  if (nact(g) == 3) k_chk_rows<3><<<gr, TPB, 0, st>>>(g, p, in, kind, D, C[0], C[1], c2, rhs, chk);
  else k_chk_rows<2><<<gr, TPB, 0, st>>>(g, p, in, kind, D, C[0], C[1], c2, rhs, chk);
}

}  // namespace dg
