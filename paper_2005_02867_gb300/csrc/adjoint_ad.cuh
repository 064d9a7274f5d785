// Local derivatives for the discrete adjoint of the step with flow.
//
// Each stage of the step computes, per cell or face, a few outputs from a small stencil of
// inputs.  Its adjoint needs sum_j w_j d(out_j)/d(in) for every input of the stencil, the
// weights w_j coming from the adjoint of the later stages.  The stage formulas are written
// once, over a value type that carries one tangent (Tan: value and derivative), with every
// input read through a counting reader (Rd).  The reader seeds the tangent of one read per
// evaluation; evaluating the formula once per read gives that read's column of the local
// Jacobian, which is weighted and added into the adjoint of the array the value came from.
// Branch decisions (upwind sides, limiter and minmod choices, clipping, pinned rows) follow
// the values, so they are those of the forward step: the derivative is that of the forward
// map with its branches held.
#pragma once
#include "common.cuh"

namespace dg {

struct Tan {
  double v, t;
};
__device__ __forceinline__ Tan tc(double v) { return Tan{v, 0.0}; }
__device__ __forceinline__ Tan operator+(Tan a, Tan b) { return Tan{a.v + b.v, a.t + b.t}; }
__device__ __forceinline__ Tan operator-(Tan a, Tan b) { return Tan{a.v - b.v, a.t - b.t}; }
__device__ __forceinline__ Tan operator-(Tan a) { return Tan{-a.v, -a.t}; }
__device__ __forceinline__ Tan operator*(Tan a, Tan b) { return Tan{a.v * b.v, a.t * b.v + a.v * b.t}; }
__device__ __forceinline__ Tan operator*(double s, Tan a) { return Tan{s * a.v, s * a.t}; }
__device__ __forceinline__ Tan operator*(Tan a, double s) { return Tan{a.v * s, a.t * s}; }
__device__ __forceinline__ Tan operator+(Tan a, double s) { return Tan{a.v + s, a.t}; }
__device__ __forceinline__ Tan operator+(double s, Tan a) { return Tan{s + a.v, a.t}; }
__device__ __forceinline__ Tan operator-(Tan a, double s) { return Tan{a.v - s, a.t}; }
__device__ __forceinline__ Tan operator-(double s, Tan a) { return Tan{s - a.v, -a.t}; }
__device__ __forceinline__ Tan operator/(Tan a, Tan b) {
  const double q = a.v / b.v;
  return Tan{q, (a.t - q * b.t) / b.v};
}
__device__ __forceinline__ Tan operator/(Tan a, double s) { return Tan{a.v / s, a.t / s}; }
__device__ __forceinline__ Tan operator/(double s, Tan b) {
  const double q = s / b.v;
  return Tan{q, -q * b.t / b.v};
}
__device__ __forceinline__ Tan tsqrt(Tan a) {
  const double r = sqrt(a.v);
  return Tan{r, r > 0.0 ? a.t / (2.0 * r) : 0.0};
}
__device__ __forceinline__ Tan tabs(Tan a) { return a.v < 0.0 ? -a : a; }
// the forward kernels' min / max (ties take the first operand) and clamp
__device__ __forceinline__ Tan tmax(Tan a, Tan b) { return ord64(a.v) >= ord64(b.v) ? a : b; }
__device__ __forceinline__ Tan tmin(Tan a, Tan b) { return ord64(a.v) <= ord64(b.v) ? a : b; }
__device__ __forceinline__ Tan tclamp01(Tan a) { return tmin(tc(1.0), tmax(tc(0.0), a)); }
// minmod: the operand of smaller magnitude when both are non-zero with the same sign
__device__ __forceinline__ Tan tminmod(Tan x, Tan y) {
  const long long bx = __double_as_longlong(x.v), by = __double_as_longlong(y.v);
  const long long ax = bx & 0x7FFFFFFFFFFFFFFFLL, ay = by & 0x7FFFFFFFFFFFFFFFLL;
  const bool same = (bx ^ by) >= 0 && ax != 0 && ay != 0;
  return same ? (ax <= ay ? x : y) : tc(0.0);
}
__device__ __forceinline__ Tan tlim_up(Tan uu, Tan u, Tan d) { return u + 0.5 * tminmod(u - uu, d - u); }
__device__ __forceinline__ Tan tvan_leer(Tan uu, Tan u, Tan d) {
  const Tan dU = u - uu, dD = d - u, pr = dU * dD;
  return pr.v > 0.0 ? u + pr / (dU + dD) : u;
}

// d Y_eq / d T for the Raoult model (0 where the mole fraction is clamped)
__device__ __forceinline__ double dYeq_dT(const Phys& p, double T) {
  double y = psat(p, T) / p.P;
  if (y > Y_CLAMP) return 0.0;
  double dy = y * (p.Lv * p.M_l / R_GAS) / (T * T);
  double den = y * p.M_l + (1.0 - y) * p.M_g;
  return dy * p.M_l * p.M_g / (den * den);
}

// Arrays whose adjoints the stage formulas scatter into, and the scalar parameters
enum AdjArr {
  J_ALPHA_N = 0,   // alpha^n
  J_T_N,           // T^n
  J_WP,            // omega' (omega^n with the liquid pinned, S0)
  J_U0, J_U1, J_U2,   // u^n, faces of each direction
  J_P_N,           // p_rgh^n
  J_ASTAR,         // alpha* (after the source)
  J_AL,            // low-order alpha^L
  J_FL0, J_FL1, J_FL2,   // low-order face fluxes
  J_AF0, J_AF1, J_AF2,   // antidiffusive face fluxes
  J_RP, J_RM,      // limiter ratios
  J_ALPHA1,        // alpha^{n+1}
  J_RHO, J_MU, J_KC, J_CP, J_DM,   // mixture properties (at alpha^{n+1})
  J_MDOT,          // evaporation rate
  J_RGO, J_RGN,    // rho_G^n, rho_G^{n+1}
  J_YQ,            // saturation value of the pinned species rows
  J_US0, J_US1, J_US2,   // u*
  J_DP,            // pressure increment
  J_COUNT,
  J_PAR_TAMB = 64, // ambient temperature (boundary values)
  J_PAR_DGAS       // gas diffusivity D_gas
};

// Counting reader: read number `seed` gets tangent 1 and its source is recorded
struct Rd {
  int seed, cnt, arr;
  long long idx;
  __device__ explicit Rd(int s) : seed(s), cnt(0), arr(-1), idx(-1) {}
  __device__ __forceinline__ Tan operator()(const double* a, int id, long long i) {
    Tan r{a[i], 0.0};
    if (cnt == seed) { r.t = 1.0; arr = id; idx = i; }
    ++cnt;
    return r;
  }
  __device__ __forceinline__ Tan par(double v, int id) {
    Tan r{v, 0.0};
    if (cnt == seed) { r.t = 1.0; arr = id; idx = -1; }
    ++cnt;
    return r;
  }
};

// Adjoint arrays by AdjArr index; parameter adjoints go to acc[AC_TAMB_BC], acc[AC_DGAS]
struct AdjT {
  double* lam[J_COUNT];
  double* acc;
};

}  // namespace dg
