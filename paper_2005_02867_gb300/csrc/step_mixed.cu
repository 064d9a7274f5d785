// Mixed-precision assembly of the momentum predictor and of the energy / species systems
// (precision 1: FP32 stencils, FP64 state).  The terms that carry the state stay FP64:
// rho V / dt and rho V u / dt for the momentum (Sec. 2.5, momentum equation), c V / dt
// and c V phi / dt, the phase-change source and the pinned rows for the scalars
// (Eqs. Teqn, speciesequation).  The per-step increments -- advection, viscous and
// diffusive fluxes, the pressure / buoyancy / centripetal forces, the couplings -- are
// formed in FP32 from inputs rounded on the integer pipe (f32_rn), differences of state
// fields taken in FP64 first, so that each rounding is relative to the increment of one
// step and not to the state.  The operations, stencils and boundary rules are those of
// k_mom_assemble and k_scalar_assemble; only the arithmetic type of the increments differs.
#include "kernels.h"

namespace dg {

struct GeoF {
  float h[3], ih[3];
};
__device__ __forceinline__ GeoF geof(const Geo& g) {
  GeoF q;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    q.h[a] = f32_rn(g.h[a]);
    q.ih[a] = f32_rn(g.ih[a]);
  }
  return q;
}

__device__ __forceinline__ float ldf(const double* p, long long i) { return f32_rn(p[i]); }
// a binary32 copy holds the rounded values already (the accessors below take either)
__device__ __forceinline__ float ldf(const float* p, long long i) { return p[i]; }

__device__ __forceinline__ float minmod_f(float x, float y) {
  return (x * y > 0.f) ? (x > 0.f ? fminf(fabsf(x), fabsf(y)) : -fminf(fabsf(x), fabsf(y))) : 0.f;
}
__device__ __forceinline__ float lim_up_f(float uu, float u, float d) { return u + 0.5f * minmod_f(u - uu, d - u); }

__device__ __forceinline__ float areaN_f(const Geo& g, const GeoF& q, int a, float rl) {
  if (g.axisym) return rl * (a == 0 ? q.h[1] : q.h[0]);
  return q.h[0] * q.h[1] * q.h[2] * q.ih[a];
}

// face velocity of direction c with ghosts (the rules of ufg), rounded to FP32
template <typename FT>
__device__ __forceinline__ float ufg_f(const Geo& g, const FT* uc, int c, int i, int j, int k) {
  int m0 = g.n[0] + (c == 0), m1 = g.n[1] + (c == 1), m2 = g.n[2] + (c == 2);
  int a, side, q, m;
  if (i < 0 || i >= m0) { a = 0; q = i; m = m0; }
  else if (j < 0 || j >= m1) { a = 1; q = j; m = m1; }
  else if (k < 0 || k >= m2) { a = 2; q = k; m = m2; }
  else return ldf(uc, fidx(g, c, i, j, k));
  side = q < 0 ? 0 : 1;
  int kind = bc_of(g, a, side);
  int kk = side ? q - (m - 1) : -q;
  int qb;
  float sign = 1.f, base = 0.f;
  if (a == c) {
    int qe = side ? m - 1 : 0;
    float ub = ldf(uc, fidx(g, c, a == 0 ? qe : i, a == 1 ? qe : j, a == 2 ? qe : k));
    if (kind == BC_OPEN) return ub;
    qb = side ? m - 1 - kk : kk;
    base = 2.f * ub;
    sign = -1.f;
  } else {
    if (kind == BC_OPEN) qb = side ? m - 1 : 0;
    else qb = side ? m - kk : kk - 1;
    sign = (kind == BC_OPEN || kind == BC_AXIS) ? 1.f : -1.f;
  }
  float v = ldf(uc, fidx(g, c, a == 0 ? qb : i, a == 1 ? qb : j, a == 2 ? qb : k));
  return base + sign * v;
}

template <typename FT>
__device__ __forceinline__ float cellc_f(const Geo& g, const FT* f, int i, int j, int k) {
  i = i < 0 ? 0 : (i >= g.n[0] ? g.n[0] - 1 : i);
  j = j < 0 ? 0 : (j >= g.n[1] ? g.n[1] - 1 : j);
  k = k < 0 ? 0 : (k >= g.n[2] ? g.n[2] - 1 : k);
  return ldf(f, cidx(g, i, j, k));
}

template <typename FT>
__device__ __forceinline__ float mu_edge_f(const Geo& g, const FT* mu, const int L[3], const int R[3], int a,
                                           int sh) {
  int La[3] = {L[0], L[1], L[2]}, Ra[3] = {R[0], R[1], R[2]};
  La[a] += sh;
  Ra[a] += sh;
  float s = cellc_f(g, mu, L[0], L[1], L[2]) + cellc_f(g, mu, R[0], R[1], R[2]) + cellc_f(g, mu, La[0], La[1], La[2]) +
            cellc_f(g, mu, Ra[0], Ra[1], Ra[2]);
  return 0.25f * s;
}

// scalar cell value with ghosts (the rules of cellg), rounded to FP32
template <typename FT>
__device__ __forceinline__ float cellg_f(const Geo& g, const FT* f, int i, int j, int k, int rule, float amb,
                                         const double* u0, const double* u1, const double* u2) {
  int a, side;
  if (i < 0) { a = 0; side = 0; i = 0; }
  else if (i >= g.n[0]) { a = 0; side = 1; i = g.n[0] - 1; }
  else if (j < 0) { a = 1; side = 0; j = 0; }
  else if (j >= g.n[1]) { a = 1; side = 1; j = g.n[1] - 1; }
  else if (k < 0) { a = 2; side = 0; k = 0; }
  else if (k >= g.n[2]) { a = 2; side = 1; k = g.n[2] - 1; }
  else return ldf(f, cidx(g, i, j, k));
  float vb = ldf(f, cidx(g, i, j, k));
  int kind = bc_of(g, a, side);
  if (rule == R_ALPHA) return kind == BC_AXIS ? vb : 0.f;
  if (rule == R_ZG) return vb;
  if (kind == BC_AXIS || kind == BC_WALL) return vb;
  if (kind == BC_FORCED) return 2.f * amb - vb;
  int fi = i, fj = j, fk = k;
  if (side) {
    if (a == 0) fi = g.n[0];
    else if (a == 1) fj = g.n[1];
    else fk = g.n[2];
  }
  const double* ua = a == 0 ? u0 : (a == 1 ? u1 : u2);
  double un = ua[fidx(g, a, fi, fj, fk)];
  double vout = side ? un : -un;
  return vout < 0.0 ? 2.f * amb - vb : vb;
}

// FIB: with the fibre (faces of its sphere pinned at u* = 0; a neighbour face's coupling to
// one of them goes into the neighbour's diagonal), as in the FP64 kernel
template <int C, int NA, bool FIB>
__global__ void __launch_bounds__(TPB, 4) k_mom_assemble_mx(Geo g, Phys p, const double* u0, const double* u1, const double* u2,
                                  const double* rho, const double* pr, const double* alpha, const double* xi,
                                  const float* muf, const float* uf0, const float* uf1, const float* uf2,
                                  double* Dg, double* c0, double* c1, double* c2, double* rhs) {
  constexpr int c = C;
  int m[3] = {g.n[0], g.n[1], g.n[2]};
  m[c] -= 1;
  long long nb = (long long)m[0] * m[1] * m[2];
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= nb) return;
  int b[3];
  decomp(id, m[0], m[1], b[0], b[1], b[2]);
  int f[3] = {b[0], b[1], b[2]};
  f[c] += 1;
  int L[3] = {f[0], f[1], f[2]}, R[3] = {f[0], f[1], f[2]};
  L[c] -= 1;
  const GeoF q = geof(g);
  const double* U[3] = {u0, u1, u2};
  const double* uc = U[c];
  const float* UF[3] = {uf0, uf1, uf2};
  const float* ucf = UF[c];
  double* Cc[3] = {c0, c1, c2};
  constexpr int na = NA;
  long long li = cidx(g, L[0], L[1], L[2]), ri = cidx(g, R[0], R[1], R[2]);
  // the state terms, FP64
  const double rhoL = rho[li], rhoR = rho[ri];
  const double rho_f = 0.5 * (rhoL + rhoR);
  double r_f = 0.0, V_f;
  if (g.axisym) {
    r_f = (c == 0) ? f[0] * g.h[0] : (f[0] + 0.5) * g.h[0];
    V_f = r_f * g.h[0] * g.h[1];
  } else {
    V_f = g.h[0] * g.h[1] * g.h[2];
  }
  const double u_f = uc[fidx(g, c, f[0], f[1], f[2])];
  const double d0 = rho_f * V_f * idt_of(p);
  if (FIB && sphere_face(g, c, f[0], f[1], f[2])) {   // a face of the sphere: a decoupled row, u* = 0
    Dg[id] = d0;
    rhs[id] = 0.0;
#pragma unroll
    for (int a = 0; a < NA; ++a) Cc[a][id] = 0.0;
    return;
  }
  // the increments, FP32
  const float rho_ff = f32_rn(rho_f), V_ff = f32_rn(V_f), r_ff = f32_rn(r_f);
  const float A_ff = V_ff * q.ih[c];
  const float muL = muf[li], muR = muf[ri];
  const float mu_f = 0.5f * (muL + muR);
  const float u_ff = ucf[fidx(g, c, f[0], f[1], f[2])];
  float t_adv = 0.f, t_vT = 0.f, d_visc = 0.f, t_bnd = 0.f;
#pragma unroll
  for (int a = 0; a < na; ++a) {
    // ---- advection (advective form, minmod limited linear upwind)
    float ubar;
    if (a == c) ubar = u_ff;
    else {
      const float* ua = UF[a];
      int La[3] = {L[0], L[1], L[2]}, Ra[3] = {R[0], R[1], R[2]};
      La[a] += 1;
      Ra[a] += 1;
      ubar = 0.25f * (((ldf(ua, fidx(g, a, L[0], L[1], L[2])) + ldf(ua, fidx(g, a, La[0], La[1], La[2]))) +
                       ldf(ua, fidx(g, a, R[0], R[1], R[2]))) + ldf(ua, fidx(g, a, Ra[0], Ra[1], Ra[2])));
    }
    int qq[3];
    float us[5];
#pragma unroll
    for (int s = -2; s <= 2; ++s) {
      qq[0] = f[0]; qq[1] = f[1]; qq[2] = f[2];
      qq[a] += s;
      us[s + 2] = ufg_f(g, ucf, c, qq[0], qq[1], qq[2]);
    }
    float uplus, uminus;
    if (ubar >= 0.f) { uplus = lim_up_f(us[1], us[2], us[3]); uminus = lim_up_f(us[0], us[1], us[2]); }
    else { uplus = lim_up_f(us[4], us[3], us[2]); uminus = lim_up_f(us[3], us[2], us[1]); }
    t_adv = t_adv - rho_ff * V_ff * ubar * (uplus - uminus) * q.ih[a];
    // ---- viscous
    if (a == c) {
      float ApL, ApR;
      if (g.axisym && c == 0) {
        ApL = areaN_f(g, q, 0, (L[0] + 0.5f) * q.h[0]);
        ApR = areaN_f(g, q, 0, (R[0] + 0.5f) * q.h[0]);
      } else if (g.axisym) {
        ApL = ApR = areaN_f(g, q, 1, r_ff);
      } else {
        ApL = ApR = areaN_f(g, q, c, 0.f);
      }
      float kR = muR * ApR * q.ih[c], kL = muL * ApL * q.ih[c];
      float dR = (us[3] - us[2]) * q.ih[c], dL = (us[2] - us[1]) * q.ih[c];
      t_vT = t_vT + muR * ApR * dR - muL * ApL * dL;
      Cc[c][id] = (b[c] > 0) ? f64_of(kL) : 0.0;
      if (b[c] == 0 && g.bc[c][0] != BC_OPEN) {
        int fb[3] = {f[0], f[1], f[2]};
        fb[c] = 0;
        d_visc += kL;
        t_bnd += kL * ucf[fidx(g, c, fb[0], fb[1], fb[2])];
      }
      if (b[c] == m[c] - 1 && g.bc[c][1] != BC_OPEN) {
        int fb[3] = {f[0], f[1], f[2]};
        fb[c] = g.n[c];
        d_visc += kR;
        t_bnd += kR * ucf[fidx(g, c, fb[0], fb[1], fb[2])];
      }
      if (FIB) {   // neighbour faces along c on the sphere
        if (b[c] > 0 && sphere_face(g, c, f[0] - (c == 0), f[1] - (c == 1), f[2] - (c == 2))) {
          Cc[c][id] = 0.0;
          d_visc += kL;
        }
        if (b[c] < m[c] - 1 && sphere_face(g, c, f[0] + (c == 0), f[1] + (c == 1), f[2] + (c == 2))) d_visc += kR;
      }
    } else {
      float App, Apm;
      if (g.axisym && a == 0) {
        App = areaN_f(g, q, 0, (f[0] + 1) * q.h[0]);
        Apm = areaN_f(g, q, 0, f[0] * q.h[0]);
      } else if (g.axisym) {
        App = Apm = areaN_f(g, q, 1, r_ff);
      } else {
        App = Apm = areaN_f(g, q, a, 0.f);
      }
      float mup = mu_edge_f(g, muf, L, R, a, 1), mum = mu_edge_f(g, muf, L, R, a, -1);
      float kp = mup * App * q.ih[a], km = mum * Apm * q.ih[a];
      const float* ua = UF[a];
      int La[3] = {L[0], L[1], L[2]}, Ra[3] = {R[0], R[1], R[2]};
      La[a] += 1;
      Ra[a] += 1;
      float uaR_hi = ldf(ua, fidx(g, a, Ra[0], Ra[1], Ra[2])), uaL_hi = ldf(ua, fidx(g, a, La[0], La[1], La[2]));
      float uaR_lo = ldf(ua, fidx(g, a, R[0], R[1], R[2])), uaL_lo = ldf(ua, fidx(g, a, L[0], L[1], L[2]));
      t_vT = t_vT + mup * App * (uaR_hi - uaL_hi) * q.ih[c] - mum * Apm * (uaR_lo - uaL_lo) * q.ih[c];
      Cc[a][id] = (b[a] > 0) ? f64_of(km) : 0.0;
      if (b[a] == 0 && (g.bc[a][0] == BC_WALL || g.bc[a][0] == BC_FORCED)) d_visc += 2.f * km;
      if (b[a] == m[a] - 1 && (g.bc[a][1] == BC_WALL || g.bc[a][1] == BC_FORCED)) d_visc += 2.f * kp;
      if (FIB) {   // neighbour faces along a on the sphere
        if (b[a] > 0 && sphere_face(g, c, f[0] - (a == 0), f[1] - (a == 1), f[2] - (a == 2))) {
          Cc[a][id] = 0.0;
          d_visc += km;
        }
        if (b[a] < m[a] - 1 && sphere_face(g, c, f[0] + (a == 0), f[1] + (a == 1), f[2] + (a == 2))) d_visc += kp;
      }
    }
  }
  if (g.axisym && c == 0 && r_ff > 0.f) d_visc = d_visc + 2.f * mu_f * V_ff / (r_ff * r_ff);
  // pressure, buoyancy and centripetal force in the balanced face form (differences in FP64)
  float gx = 0.f;
#pragma unroll
  for (int a = 0; a < na; ++a) {
    float xa = (a == c) ? f[a] * q.h[a] : (f[a] + 0.5f) * q.h[a];
    gx = gx + f32_rn(p.g[a]) * xa;
  }
  const float dpr = f32_rn(pr[ri] - pr[li]), drho = f32_rn(rhoR - rhoL), dxi = f32_rn(xi[ri] - xi[li]);
  const float raL = f32_rn(rhoL * alpha[li]), raR = f32_rn(rhoR * alpha[ri]);
  const float t_force = -A_ff * dpr - A_ff * gx * drho + A_ff * 0.5f * (raL + raR) * dxi;
  Dg[id] = d0 + f64_of(d_visc);
  rhs[id] = d0 * u_f + f64_of(((t_adv + t_vT) + t_force) + t_bnd);
}

// FIB: with the fibre (its cells carry gamma = 0; the harmonic mean of two zeros is 0, and a
// far upwind value inside it is replaced by the near one).  HD (energy rows, c_p,v != c_p,g):
// the species-diffusion enthalpy term of Eq. Teqn as in the FP64 kernel, formed in binary32
// from the copies of rho D (gdf) and omega^n (wf) as one more increment
template <int NA, bool FIB, bool HD = false>
// phif, gf, uf*: binary32 copies of phi, of gamma (k, or rho D) and of the face velocities
__global__ void k_scalar_assemble_mx(Geo g, Phys p, int mode, const double* phi, const double* rho, const double* cp,
                                     const double* mdot, const double* u0, const double* u1, const double* u2,
                                     const double* alpha_new, const double* pinv, double amb, const float* phif,
                                     const float* gf, const float* uf0, const float* uf1, const float* uf2,
                                     double* Dg, double* c0, double* c1, double* c2, double* rhs,
                                     const float* gdf, const float* wf) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  int i, j, k;
  decomp(id, g.n[0], g.n[1], i, j, k);
  constexpr int na = NA;
  const GeoF q = geof(g);
  const double* U[3] = {u0, u1, u2};
  const float* UF[3] = {uf0, uf1, uf2};
  double* C[3] = {c0, c1, c2};
  // the state terms, FP64 (storage c V / dt and its phi term, the phase-change source)
  const double V = cellV(g, i);
  const double coef = mode == 0 ? rho[id] * cp[id] : rho[id];
  double dP = coef * V * idt_of(p);
  double r = coef * V * phi[id] * idt_of(p) + (mode == 0 ? -mdot[id] * p.Lv : 0.0) * V;
  const bool pin = (mode == 1) && ige64(alpha_new[id], 0.5);
  // the increments, FP32
  const float phiP = phif[id], ambf = f32_rn(amb);
  const float gP = gf[id];
  float net = 0.f, Fsum = 0.f, dinc = 0.f, rinc = 0.f;
  int ci[3] = {i, j, k};
  float hq = 0.f, gdP = 0.f, wP = 0.f;   // HD: the face sum, rho D and omega of the cell
  if (HD) {
    gdP = gdf[id];
    wP = wf[id];
  }
#pragma unroll
  for (int a = 0; a < na; ++a) {
    if (HD) {
      if (ci[a] > 0) {
        int Lc[3] = {i, j, k};
        Lc[a] -= 1;
        const long long li = cidx(g, Lc[0], Lc[1], Lc[2]);
        const float gL = gdf[li];
        const float Aa = a == 0 ? (g.axisym ? (i * q.h[0]) * q.h[1] : q.h[0] * q.h[1] * q.h[2] * q.ih[0])
                                : (g.axisym ? ((i + 0.5f) * q.h[0]) * q.h[0] : q.h[0] * q.h[1] * q.h[2] * q.ih[a]);
        const float cf = (FIB && gL + gdP == 0.f) ? 0.f : 2.f * gL * gdP / (gL + gdP) * Aa * q.ih[a];
        hq += cf * (wf[li] - wP) * (phif[li] - phiP);
      }
      if (ci[a] < g.n[a] - 1) {
        int Hc[3] = {i, j, k};
        Hc[a] += 1;
        const long long hi = cidx(g, Hc[0], Hc[1], Hc[2]);
        const float gH = gdf[hi];
        const float Ah = a == 0 ? (g.axisym ? (Hc[0] * q.h[0]) * q.h[1] : q.h[0] * q.h[1] * q.h[2] * q.ih[0])
                                : (g.axisym ? ((i + 0.5f) * q.h[0]) * q.h[0] : q.h[0] * q.h[1] * q.h[2] * q.ih[a]);
        const float cf = (FIB && gdP + gH == 0.f) ? 0.f : 2.f * gdP * gH / (gdP + gH) * Ah * q.ih[a];
        hq += cf * (wf[hi] - wP) * (phif[hi] - phiP);
      }
    }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      int f[3] = {i, j, k};
      if (side) f[a] += 1;
      const float Af = a == 0 ? (g.axisym ? (f[0] * q.h[0]) * q.h[1] : q.h[0] * q.h[1] * q.h[2] * q.ih[0])
                              : (g.axisym ? ((f[0] + 0.5f) * q.h[0]) * q.h[0] : q.h[0] * q.h[1] * q.h[2] * q.ih[a]);
      const float F = UF[a][fidx(g, a, f[0], f[1], f[2])] * Af;
      float val;
      if (f[a] == 0 || f[a] == g.n[a]) {
        int kind = (side ? g.bc[a][1] : g.bc[a][0]);
        bool inflow = side == 0 ? (F > 0.f) : (F < 0.f);
        val = ((kind == BC_OPEN || kind == BC_FORCED) && inflow) ? ambf : phiP;
      } else {
        int Lc[3] = {f[0], f[1], f[2]};
        Lc[a] -= 1;
        int LL[3] = {Lc[0], Lc[1], Lc[2]}, RR[3] = {f[0], f[1], f[2]};
        LL[a] -= 1;
        RR[a] += 1;
        float vL = phif[cidx(g, Lc[0], Lc[1], Lc[2])], vR = phif[cidx(g, f[0], f[1], f[2])];
        if (F >= 0.f) {
          const float far = FIB && solid_nb(g, LL[0], LL[1], LL[2]) ? vL : cellg_f(g, phif, LL[0], LL[1], LL[2], R_TO, ambf, u0, u1, u2);
          val = lim_up_f(far, vL, vR);
        } else {
          const float far = FIB && solid_nb(g, RR[0], RR[1], RR[2]) ? vR : cellg_f(g, phif, RR[0], RR[1], RR[2], R_TO, ambf, u0, u1, u2);
          val = lim_up_f(far, vR, vL);
        }
      }
      // advected value relative to the cell's own: the flux difference then carries
      // only the increment (net - phi Fsum of the FP64 form, without its cancellation)
      const float sgn = side ? 1.f : -1.f;
      net += sgn * F * (val - phiP);
      Fsum += sgn * F;
    }
    // coupling across the low face, stored at this cell
    float cl = 0.f;
    if (ci[a] > 0) {
      int Lc[3] = {i, j, k};
      Lc[a] -= 1;
      long long li = cidx(g, Lc[0], Lc[1], Lc[2]);
      const float gL = gf[li];
      const float Aa = a == 0 ? (g.axisym ? (i * q.h[0]) * q.h[1] : q.h[0] * q.h[1] * q.h[2] * q.ih[0])
                              : (g.axisym ? ((i + 0.5f) * q.h[0]) * q.h[0] : q.h[0] * q.h[1] * q.h[2] * q.ih[a]);
      cl = (FIB && gL + gP == 0.f) ? 0.f : 2.f * gL * gP / (gL + gP) * Aa * q.ih[a];
      if (mode == 1) {
        bool lp = ige64(alpha_new[li], 0.5);
        if (!pin && lp) { r += f64_of(cl) * pinv[li]; dinc += cl; }
        if (pin || lp) cl = 0.f;
      }
    }
    C[a][id] = f64_of(cl);
    // coupling across the high face (owned by the neighbour): only the pinned-neighbour transfer here
    if (mode == 1 && ci[a] < g.n[a] - 1 && !pin) {
      int Hc[3] = {i, j, k};
      Hc[a] += 1;
      long long hi = cidx(g, Hc[0], Hc[1], Hc[2]);
      if (ige64(alpha_new[hi], 0.5)) {
        const float gH = gf[hi];
        const float Ah = a == 0 ? (g.axisym ? (Hc[0] * q.h[0]) * q.h[1] : q.h[0] * q.h[1] * q.h[2] * q.ih[0])
                                : (g.axisym ? ((i + 0.5f) * q.h[0]) * q.h[0] : q.h[0] * q.h[1] * q.h[2] * q.ih[a]);
        const float ch = (FIB && gP + gH == 0.f) ? 0.f : 2.f * gP * gH / (gP + gH) * Ah * q.ih[a];
        r += f64_of(ch) * pinv[hi];
        dinc += ch;
      }
    }
    // Dirichlet boundary faces
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      bool atb = side ? (ci[a] == g.n[a] - 1) : (ci[a] == 0);
      if (!atb) continue;
      int kind = (side ? g.bc[a][1] : g.bc[a][0]);
      bool isdir = false;
      int f[3] = {i, j, k};
      if (side) f[a] += 1;
      if (kind == BC_FORCED) isdir = true;
      else if (kind == BC_OPEN) {
        double un = U[a][fidx(g, a, f[0], f[1], f[2])];
        isdir = (side ? un : -un) < 0.0;
      }
      if (isdir) {
        const float Ab = a == 0 ? (g.axisym ? (f[0] * q.h[0]) * q.h[1] : q.h[0] * q.h[1] * q.h[2] * q.ih[0])
                                : (g.axisym ? ((i + 0.5f) * q.h[0]) * q.h[0] : q.h[0] * q.h[1] * q.h[2] * q.ih[a]);
        const float cb = gP * Ab * (2.f * q.ih[a]);
        dinc += cb;
        rinc += cb * (ambf - phiP);   // relative to phi: the cb phi part is added in FP64 below
        r += f64_of(cb) * phi[id];
      }
    }
  }
  if (HD) rinc += 0.5f * f32_rn(p.cp_v - p.cp_g) * hq;
  // - coef (net - phi Fsum): the FP32 sum above is already relative to phi
  r += f64_of(rinc) - coef * f64_of(net);
  dP += f64_of(dinc);
  if (pin) {
    // pinned row, scaled like the other rows: (coef V/dt) x = (coef V/dt) Y_eq
    double dd = coef * V * idt_of(p);
    r = dd * pinv[id];
    dP = dd;
  }
  Dg[id] = dP;
  rhs[id] = r;
}

// alpha of a cell or ghost from its binary32 copy, with the ghost rule of alpha (the
// axis mirrors, every other boundary has alpha = 0 outside): cellg_f(..., R_ALPHA, ...)
// of the binary64 field, without a rounding per reference
__device__ __forceinline__ float alpha_gf(const Geo& g, const float* f, int i, int j, int k) {
  int a, side;
  if (i < 0) { a = 0; side = 0; i = 0; }
  else if (i >= g.n[0]) { a = 0; side = 1; i = g.n[0] - 1; }
  else if (j < 0) { a = 1; side = 0; j = 0; }
  else if (j >= g.n[1]) { a = 1; side = 1; j = g.n[1] - 1; }
  else if (k < 0) { a = 2; side = 0; k = 0; }
  else if (k >= g.n[2]) { a = 2; side = 1; k = g.n[2] - 1; }
  else return f[cidx(g, i, j, k)];
  return bc_of(g, a, side) == BC_AXIS ? f[cidx(g, i, j, k)] : 0.f;
}

// alpha gradient of a cell (central differences, the ghost rule of alpha), FP32
// (a neighbour inside the fibre takes the cell's own value: zero gradient across the sphere)
__device__ __forceinline__ float alpha_gf_m(const Geo& g, const float* f, int i, int j, int k, int ni, int nj, int nk) {
  return solid_nb(g, ni, nj, nk) ? f[cidx(g, i, j, k)] : alpha_gf(g, f, ni, nj, nk);
}
__device__ __forceinline__ void grad_alpha_f(const Geo& g, const GeoF& q, const float* al, int i, int j, int k,
                                             float gr[3]) {
  if (g.fib) {
    gr[0] = (alpha_gf_m(g, al, i, j, k, i + 1, j, k) - alpha_gf_m(g, al, i, j, k, i - 1, j, k)) * (0.5f * q.ih[0]);
    gr[1] = (alpha_gf_m(g, al, i, j, k, i, j + 1, k) - alpha_gf_m(g, al, i, j, k, i, j - 1, k)) * (0.5f * q.ih[1]);
    gr[2] = g.act3 ? (alpha_gf_m(g, al, i, j, k, i, j, k + 1) - alpha_gf_m(g, al, i, j, k, i, j, k - 1)) * (0.5f * q.ih[2])
                   : 0.f;
    return;
  }
  gr[0] = (alpha_gf(g, al, i + 1, j, k) - alpha_gf(g, al, i - 1, j, k)) * (0.5f * q.ih[0]);
  gr[1] = (alpha_gf(g, al, i, j + 1, k) - alpha_gf(g, al, i, j - 1, k)) * (0.5f * q.ih[1]);
  gr[2] = g.act3 ? (alpha_gf(g, al, i, j, k + 1) - alpha_gf(g, al, i, j, k - 1)) * (0.5f * q.ih[2]) : 0.f;
}

// Face fluxes of the alpha advection (Sec. 2.1 with the compressive flux), mixed
// precision: the low-order upwind flux phi alpha_up stays FP64 (it decides the bounds
// of the low-order solution); the antidiffusive flux A = FH - FL is formed directly as
// phi (van Leer increment) + C_alpha |phi| (n_f . e) a_c (1 - a_c) in FP32 -- equal to
// the difference in exact arithmetic, without its cancellation.  Fluxes are applied
// antisymmetrically, so the volume stays conserved whatever their precision, and the
// limiter bounds the result as in k_adv_faces.  The FP32 stencil reads alpha* from its
// binary32 copy asf.
template <int DIR, int NA>
__device__ __forceinline__ void adv_face_mx(const Geo& g, const Phys& p, const double* as, const float* asf,
                                            const double* ua, double* FL, double* AF, long long id) {
  constexpr int a = DIR;
  int m0 = g.n[0] + (a == 0), m1 = g.n[1] + (a == 1);
  int f[3];
  decomp(id, m0, m1, f[0], f[1], f[2]);
  int L[3] = {f[0], f[1], f[2]}, R[3] = {f[0], f[1], f[2]};
  L[a] -= 1;
  const double phi = ua[id] * faceA(g, a, f[0]) * dt_of(p);
  const double aL = cellg(g, as, L[0], L[1], L[2], R_ALPHA, 0, 0, 0, 0);
  const double aR = cellg(g, as, R[0], R[1], R[2], R_ALPHA, 0, 0, 0, 0);
  const bool pos = phi >= 0.0;
  FL[id] = phi * (pos ? aL : aR);
  float A = 0.f;
  // two cells of the same pure phase: no antidiffusive flux (as in the FP64 kernel)
  if (f[a] > 0 && f[a] < g.n[a] && !pure_pair(aL, aR)) {
    const GeoF q = geof(g);
    int LL[3] = {L[0], L[1], L[2]}, RR[3] = {R[0], R[1], R[2]};
    LL[a] -= 1;
    RR[a] += 1;
    const float aLf = alpha_gf(g, asf, L[0], L[1], L[2]), aRf = alpha_gf(g, asf, R[0], R[1], R[2]);
    const float aLL = alpha_gf(g, asf, LL[0], LL[1], LL[2]);
    const float aRR = alpha_gf(g, asf, RR[0], RR[1], RR[2]);
    // van Leer increment over the upwind value
    const float dU = pos ? aLf - aLL : aRf - aRR, dD = pos ? aRf - aLf : aLf - aRf, pr = dU * dD;
    const float inc = pr > 0.f ? pr / (dU + dD) : 0.f;
    float gL[3], gR[3];
    grad_alpha_f(g, q, asf, L[0], L[1], L[2], gL);
    grad_alpha_f(g, q, asf, R[0], R[1], R[2], gR);
    const float gf[3] = {gL[0] + gR[0], gL[1] + gR[1], gL[2] + gR[2]};
    const float gfm = sqrtf(gf[0] * gf[0] + gf[1] * gf[1] + (g.act3 ? gf[2] * gf[2] : 0.f));
    const float ne = gfm > f32_rn(g.gthr) ? gf[a] / gfm : 0.f;
    const float ac = 0.5f * (aLf + aRf);
    const float phif = f32_rn(phi);
    A = phif * inc + f32_rn(p.C_alpha) * fabsf(phif) * ne * ac * (1.f - ac);
  }
  AF[id] = f64_of(A);
}

// the faces of every direction in one launch: blocks [b[d], b[d + 1]) take direction d
struct AdvFacesArgs {
  const double* ua[3];
  double *FL[3], *AF[3];
  int b[4];
};
template <int NA>
__global__ void k_adv_faces_mx(Geo g, Phys p, const double* as, const float* asf, AdvFacesArgs f) {
  const int bx = blockIdx.x;
  if (bx < f.b[1]) {
    const long long id = (long long)(bx - f.b[0]) * blockDim.x + threadIdx.x;
    if (id < nfaces(g, 0)) adv_face_mx<0, NA>(g, p, as, asf, f.ua[0], f.FL[0], f.AF[0], id);
  } else if (bx < f.b[2]) {
    const long long id = (long long)(bx - f.b[1]) * blockDim.x + threadIdx.x;
    if (id < nfaces(g, 1)) adv_face_mx<1, NA>(g, p, as, asf, f.ua[1], f.FL[1], f.AF[1], id);
  } else if (NA == 3) {
    const long long id = (long long)(bx - f.b[2]) * blockDim.x + threadIdx.x;
    if (id < nfaces(g, 2)) adv_face_mx<2, NA>(g, p, as, asf, f.ua[2], f.FL[2], f.AF[2], id);
  }
}

void L_adv_faces_mx_all(cudaStream_t st, Geo g, Phys p, const double* as, const float* asf, double* const u[3],
                        double* const FL[3], double* const AF[3]) {
  AdvFacesArgs f;
  const int na = nact(g);
  int b = 0;
  for (int c = 0; c < 3; ++c) {
    f.b[c] = b;
    f.ua[c] = u[c];
    f.FL[c] = FL[c];
    f.AF[c] = AF[c];
    if (c < na) b += lin_grid(nfaces(g, c));
  }
  f.b[3] = b;
  ++g_launches;
  if (na == 3) k_adv_faces_mx<3><<<b, TPB, 0, st>>>(g, p, as, asf, f);
  else k_adv_faces_mx<2><<<b, TPB, 0, st>>>(g, p, as, asf, f);
}

void L_scalar_assemble_mx(cudaStream_t st, int grid, Geo g, Phys p, int mode, const double* phi,
                          const double* rho, const double* cp, const double* kc, const double* D, const double* mdot,
                          const double* u0, const double* u1, const double* u2, const double* alpha_new,
                          const double* pinv, double amb, double* Dg, double* c0, double* c1, double* c2, double* rhs,
                          const Shadow32* s32, const double* wq) {
  // kc and D enter through their binary32 copies (gamma = k or rho D, formed with the
  // properties); phi's copy is that of the step's old T or omega
  (void)kc;
  (void)D;
  const float* phif = mode == 0 ? s32->T : s32->w;
  const float* gf = mode == 0 ? s32->k : s32->gD;
  const float* uf2 = s32->u[2] ? s32->u[2] : s32->u[0];
  // the enthalpy term of the energy rows (wq given: omega^n, whose binary32 copy enters) when
  // the heat capacities differ
  const bool hd = mode == 0 && wq && p.cp_v != p.cp_g;
  const float* gdf = hd ? s32->gD : nullptr;
  const float* wf = hd ? s32->w : nullptr;
  ++g_launches;
#define DG_SCA(NN, FF, HH) k_scalar_assemble_mx<NN, FF, HH><<<grid, TPB, 0, st>>>(g, p, mode, phi, rho, cp, mdot, u0, u1, \
      u2, alpha_new, pinv, amb, phif, gf, s32->u[0], s32->u[1], uf2, Dg, c0, c1, c2, rhs, gdf, wf)
  if (hd) {
    if (nact(g) == 3) { if (g.fib) DG_SCA(3, true, true); else DG_SCA(3, false, true); }
    else { if (g.fib) DG_SCA(2, true, true); else DG_SCA(2, false, true); }
  } else {
    if (nact(g) == 3) { if (g.fib) DG_SCA(3, true, false); else DG_SCA(3, false, false); }
    else { if (g.fib) DG_SCA(2, true, false); else DG_SCA(2, false, false); }
  }
#undef DG_SCA
}

void L_mom_assemble_mx(cudaStream_t st, int grid, Geo g, Phys p, int c, const double* u0,
                       const double* u1, const double* u2, const double* rho, const double* mu, const double* pr,
                       const double* alpha, const double* xi, double* Dg, double* c0, double* c1, double* c2,
                       double* rhs, const Shadow32* s32) {
  (void)mu;   // through its binary32 copy
  const float *m32 = s32->mu, *f0 = s32->u[0], *f1 = s32->u[1], *f2 = s32->u[2] ? s32->u[2] : s32->u[0];
  ++g_launches;
#define DG_MOM(CC, NN, FF) k_mom_assemble_mx<CC, NN, FF><<<grid, TPB, 0, st>>>(g, p, u0, u1, u2, rho, pr, alpha, xi, m32, \
      f0, f1, f2, Dg, c0, c1, c2, rhs)
  if (nact(g) == 3) {
    if (g.fib) {
      if (c == 0) DG_MOM(0, 3, true); else if (c == 1) DG_MOM(1, 3, true); else DG_MOM(2, 3, true);
    } else {
      if (c == 0) DG_MOM(0, 3, false); else if (c == 1) DG_MOM(1, 3, false); else DG_MOM(2, 3, false);
    }
  } else {
    if (g.fib) {
      if (c == 0) DG_MOM(0, 2, true); else DG_MOM(1, 2, true);
    } else {
      if (c == 0) DG_MOM(0, 2, false); else DG_MOM(1, 2, false);
    }
  }
#undef DG_MOM
}

// the conversions themselves, for checking them against IEEE 754 rounding
__global__ void k_round_f32(const double* in, float* out32, double* back64, long long n) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= n) return;
  const float f = f32_rn(in[id]);
  out32[id] = f;
  back64[id] = f64_of(f);
}

__global__ void k_rcp64(const double* in, double* out, long long n) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= n) return;
  out[id] = rcp64(in[id]);
}

// Binary64 FMA throughput: eight independent chains per thread (enough to cover the
// FP64 pipe's latency), every SM filled; the sums are stored so that no chain is dead.
__global__ void __launch_bounds__(256) k_fma64(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = 1e-3 * threadIdx.x + q;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = fma(x[q], a, b);
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += x[q];
  out[blockIdx.x * (long long)blockDim.x + threadIdx.x] = s;
}

}  // namespace dg

extern "C" int droplet_fp64_rate(double* tflops) {
  using namespace dg;
  if (!tflops) return DROPLET_ERR_ARG;
  int dev = 0, nsm = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fma64, 256, 0) != cudaSuccess)
    return DROPLET_ERR_CUDA;
  const int blocks = nsm * (per > 0 ? per : 1), iters = 4096;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * (size_t)blocks * 256) != cudaSuccess) return DROPLET_ERR_NOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = 0;
  float best = 0.f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = DROPLET_ERR_CUDA;
  for (int rep = 0; rep < 6 && !rc; ++rep) {   // the first launch warms up; the best of the others
    cudaEventRecord(e0, 0);
    ++g_launches;
    k_fma64<<<blocks, 256>>>(out, iters, 0.999999999, 1e-9);
    cudaEventRecord(e1, 0);
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { rc = DROPLET_ERR_CUDA; break; }
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (!rc) *tflops = 2.0 * 8.0 * iters * (double)blocks * 256.0 / (best * 1e-3) / 1e12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}

extern "C" int droplet_round_f32(const double* in, float* out32, double* back64, size_t n) {
  using namespace dg;
  if (n == 0) return 0;
  if (!in || !out32 || !back64 || n > ((size_t)1 << 30)) return DROPLET_ERR_ARG;
  double *din = nullptr, *dback = nullptr;
  float* dout = nullptr;
  int rc = 0;
  if (cudaMalloc(&din, n * sizeof(double)) != cudaSuccess || cudaMalloc(&dback, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dout, n * sizeof(float)) != cudaSuccess) {
    rc = DROPLET_ERR_NOMEM;
  } else if (cudaMemcpy(din, in, n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    rc = DROPLET_ERR_CUDA;
  } else {
    ++g_launches;
    k_round_f32<<<(unsigned)((n + TPB - 1) / TPB), TPB>>>(din, dout, dback, (long long)n);
    if (cudaGetLastError() != cudaSuccess || cudaMemcpy(out32, dout, n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(back64, dback, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = DROPLET_ERR_CUDA;
  }
  cudaFree(din);
  cudaFree(dback);
  cudaFree(dout);
  return rc;
}

extern "C" int droplet_rcp_f64(const double* in, double* out, size_t n) {
  using namespace dg;
  if (n == 0) return 0;
  if (!in || !out || n > ((size_t)1 << 30)) return DROPLET_ERR_ARG;
  double *din = nullptr, *dout = nullptr;
  int rc = 0;
  if (cudaMalloc(&din, n * sizeof(double)) != cudaSuccess || cudaMalloc(&dout, n * sizeof(double)) != cudaSuccess) {
    rc = DROPLET_ERR_NOMEM;
  } else if (cudaMemcpy(din, in, n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    rc = DROPLET_ERR_CUDA;
  } else {
    ++g_launches;
    k_rcp64<<<(unsigned)((n + TPB - 1) / TPB), TPB>>>(din, dout, (long long)n);
    if (cudaGetLastError() != cudaSuccess || cudaMemcpy(out, dout, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = DROPLET_ERR_CUDA;
  }
  cudaFree(din);
  cudaFree(dout);
  return rc;
}
