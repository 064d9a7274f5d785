// Device-side definitions shared by the kernels of the droplet step:
// grid geometry, boundary rules, thermodynamics and block reductions.
//
// Grid: uniform cells, cell (i, j, k) at linear index i + n0 (j + n1 k).
// Axisymmetric runs (axisym = 1): axis 0 = r, axis 1 = z, n2 = 1, all
// volumes and areas per radian.  A face array of direction a has n_a + 1
// entries along a.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "droplet.h"

namespace dg {

enum { BC_AXIS = 0, BC_WALL = 1, BC_OPEN = 2, BC_FORCED = 3 };
enum { R_ALPHA = 0, R_ZG = 1, R_TO = 2 };

constexpr double R_GAS = 8.314462618;
constexpr double P_ATM = 101325.0;
constexpr double Y_CLAMP = 1.0 - 1e-6;
constexpr double ALPHA_GAS = 1e-3;
constexpr int RED_BLOCKS = 1216;       // 8 x 152 SMs: grid of the reduction kernels
constexpr int TPB = 256;

struct Geo {
  int n[3];
  int axisym;
  int act3;          // 1 when axis 2 is active (3D)
  int s;             // streamwise axis (gravity / inflow): 1 axisym, 2 in 3D
  int bc[3][2];
  double h[3];
  double ih[3];      // 1 / h
  double hmin;
  double gthr;       // 1e-8 / h_min: |grad alpha| above it marks an interface cell
  double vol3;       // 3D: cell volume h0 h1 h2, and face areas vol3 / h_a, formed on the host in
  double area3[3];   // the order the kernels used (the same values, no FP64 work per reference)
  // 3D momentum assembly constants, formed on the host: half the cell volume, area3[a] / h_a,
  // 0.25 area3[a] / h_a and 0.25 area3[a] / h_c (the quarter of the edge viscosity's mean
  // folded in; a product with a power of two is exact)
  double hvol3, aih[3], aih2[3], qaih[3], qvt[3][3];   // aih2 = 2 area3[a] / h_a
  double qih[3];     // 0.25 / h_a: the mean of four face velocities folded into the advection
  // gravity potential g . x at a face of direction c: gxc[c] + sum over the axes a of gmask
  // (those with g_a != 0) of gh[a] f_a, f the face's integer coordinates, gh[a] = g_a h_a,
  // gxc[c] = sum over a != c of g_a h_a / 2
  double gh[3], gxc[3];
  int gmask;
  // the spherical fibre (Table tableboundary, "sphere" row): fib = 1 with solid, one byte
  // per cell, 1 for the cells whose centre lies closer than D_f to the droplet centre
  int fib;
  const unsigned char* solid;
  int fib_lo[3], fib_hi[3];   // the box of the solid cells (inclusive cell indices)
  long long N;       // number of cells (< 2^31)
};

// Physical parameters used on the device (copied from droplet_config).
struct Phys {
  double D0, T_drop, T_amb, P, g[3], u_in, xc[3];
  double Tb, Lv, M_l, rho_l, cp_l, k_l, mu_l, D_l;
  double M_g, cp_g, cp_v, k_g, mu_g, D_g;
  double Tc, Pc, om, Tc_g, Pc_g, om_g, kij;
  double xi0, Df, dt, C_alpha, T_perturb;
  double idt;          // 1 / dt
  double D_gas;        // D_g scaled to the operating pressure
  double rhoG_const;   // frozen gas density of the constant-property check
  unsigned long long seed;
  int eq_model, const_props, physics;
  // Peng-Robinson constants of the fuel (0) and the inert gas (1), formed on the host:
  // a_c = 0.45724 R^2 Tc^2 / Pc, b = 0.07780 R Tc / Pc, kappa(omega), 1 / Tc, and
  // sqrt(a_c0 a_c1) (1 - k_ij); inverse molar masses
  double pr_ac[2], pr_b[2], pr_k[2], pr_siTc[2], pr_sqac01;   // pr_siTc = sqrt(1 / Tc)
  double iM_l, iM_g;
  // Clausius-Clapeyron exponent L M_l / R and 1 / T_b; 1 / rho_l
  double cc_LMR, iTb, irho_l;
  double drl;                // d rho_L / dT (0: constant liquid density rho_l)
  // Courant-adaptive step: the droplet's device scalars, where the step's dt and 1 / dt
  // are kept (null: the fixed dt, idt above); co_hmin = threshold Courant number x h_min
  const double* dyn;
  double co_hmin;
};

__host__ __device__ inline int nact(const Geo& g) { return g.act3 ? 3 : 2; }

// cell and face indices in 32-bit arithmetic: every array here has fewer than 2^31
// entries (cells and faces of a direction; checked when a context is created)
__device__ __forceinline__ long long cidx(const Geo& g, int i, int j, int k) {
  return (long long)(i + g.n[0] * (j + g.n[1] * k));
}
// face of direction a at integer face coords (i, j, k)
__device__ __forceinline__ long long fidx(const Geo& g, int a, int i, int j, int k) {
  const int f0 = g.n[0] + (a == 0), f1 = g.n[1] + (a == 1);
  return (long long)(i + f0 * (j + f1 * k));
}
__host__ __device__ inline long long nfaces(const Geo& g, int a) {
  return (long long)(g.n[0] + (a == 0)) * (g.n[1] + (a == 1)) * (g.n[2] + (a == 2));
}
// linear index -> (i, j, k); 32-bit arithmetic (every array here has fewer than 2^31 entries)
__device__ __forceinline__ void decomp(long long id, int n0, int n1, int& i, int& j, int& k) {
  unsigned u = (unsigned)id;
  unsigned t = u / (unsigned)n0;
  i = (int)(u - t * (unsigned)n0);
  unsigned t2 = t / (unsigned)n1;
  j = (int)(t - t2 * (unsigned)n1);
  k = (int)t2;
}

__device__ __forceinline__ double rc(const Geo& g, int i) { return (i + 0.5) * g.h[0]; }
__device__ __forceinline__ double cellV(const Geo& g, int i) {
  return g.axisym ? rc(g, i) * g.h[0] * g.h[1] : g.vol3;
}
// area of the face of direction a whose low-side cell index along 0 is i
// (for a = 0, i is the face index)
__device__ __forceinline__ double faceA(const Geo& g, int a, int i) {
  if (g.axisym) return a == 0 ? (i * g.h[0]) * g.h[1] : rc(g, i) * g.h[0];
  return g.area3[a];
}
// area of a face normal to a located at radial coordinate rl (control volumes of the momentum)
__device__ __forceinline__ double areaN(const Geo& g, int a, double rl) {
  if (g.axisym) return rl * (a == 0 ? g.h[1] : g.h[0]);
  return g.area3[a];
}

// ------------------------------------------------------------------ the fibre
// A cell of the fibre: closed to every flux, holding no fluid (zero-gradient and no-slip
// conditions on the sphere's faces).  All tests are false without a fibre (g.fib = 0).
__device__ __forceinline__ bool solid_cell(const Geo& g, long long id) { return g.fib && g.solid[id]; }
// cell (i, j, k), possibly outside the domain (then not solid)
// (the box of the solid cells first: integer compares, and the mask read only inside it)
__device__ __forceinline__ bool solid_nb(const Geo& g, int i, int j, int k) {
  return g.fib && (unsigned)(i - g.fib_lo[0]) <= (unsigned)(g.fib_hi[0] - g.fib_lo[0]) &&
         (unsigned)(j - g.fib_lo[1]) <= (unsigned)(g.fib_hi[1] - g.fib_lo[1]) &&
         (unsigned)(k - g.fib_lo[2]) <= (unsigned)(g.fib_hi[2] - g.fib_lo[2]) && g.solid[cidx(g, i, j, k)];
}
// a face of the sphere: face (i, j, k) of direction a (cells i - e_a and i) with a fibre cell
// on either side
__device__ __forceinline__ bool sphere_face(const Geo& g, int a, int i, int j, int k) {
  if (!g.fib) return false;
  return solid_nb(g, i - (a == 0), j - (a == 1), k - (a == 2)) || solid_nb(g, i, j, k);
}

// ------------------------------------------------------------------ ghosts
// Cell field value with at most one index outside the domain (by 1 or 2).
//   R_ALPHA: mirror at the axis, 0 outside other boundaries
//   R_ZG   : zero gradient (mirror at the axis)
//   R_TO   : T / omega: axis mirror, wall zero gradient, forced inlet fixed amb,
//            open boundary inletOutlet (fixed amb where the boundary face
//            velocity points inward, zero gradient otherwise)
// A fixed face value amb gives the ghost 2 amb - phi_b.
__device__ __forceinline__ int bc_of(const Geo& g, int a, int side) {
  int lo = a == 0 ? g.bc[0][0] : (a == 1 ? g.bc[1][0] : g.bc[2][0]);
  int hi = a == 0 ? g.bc[0][1] : (a == 1 ? g.bc[1][1] : g.bc[2][1]);
  return side ? hi : lo;
}

__device__ __forceinline__ double cellg(const Geo& g, const double* f, int i, int j, int k, int rule, double amb,
                                        const double* u0, const double* u1, const double* u2) {
  int a, side;
  if (i < 0) { a = 0; side = 0; i = 0; }
  else if (i >= g.n[0]) { a = 0; side = 1; i = g.n[0] - 1; }
  else if (j < 0) { a = 1; side = 0; j = 0; }
  else if (j >= g.n[1]) { a = 1; side = 1; j = g.n[1] - 1; }
  else if (k < 0) { a = 2; side = 0; k = 0; }
  else if (k >= g.n[2]) { a = 2; side = 1; k = g.n[2] - 1; }
  else return f[cidx(g, i, j, k)];
  double vb = f[cidx(g, i, j, k)];
  int kind = bc_of(g, a, side);
  if (rule == R_ALPHA) return kind == BC_AXIS ? vb : 0.0;
  if (rule == R_ZG) return vb;
  if (kind == BC_AXIS || kind == BC_WALL) return vb;
  if (kind == BC_FORCED) return 2.0 * amb - vb;
  // open boundary: the boundary face of direction a next to the clamped cell
  int fi = i, fj = j, fk = k;
  if (side) {
    if (a == 0) fi = g.n[0];
    else if (a == 1) fj = g.n[1];
    else fk = g.n[2];
  }
  const double* ua = a == 0 ? u0 : (a == 1 ? u1 : u2);
  double un = ua[fidx(g, a, fi, fj, fk)];
  double vout = side ? un : -un;
  return vout < 0.0 ? 2.0 * amb - vb : vb;
}

// Face velocity of direction c with at most one index outside its array
// (by 1 or 2).  Own axis, beyond the boundary face value u_b: axis / wall /
// forced inlet give u(-k) = 2 u_b - u(k); open boundary u(-k) = u_b.
// Tangential axis beyond the boundary cells: wall / forced inlet u(-k) =
// -u(k-1); axis u(-k) = u(k-1); open u(-k) = u(0).
__device__ __forceinline__ double ufg(const Geo& g, const double* uc, int c, int i, int j, int k) {
  int m0 = g.n[0] + (c == 0), m1 = g.n[1] + (c == 1), m2 = g.n[2] + (c == 2);
  int a, side, q, m;
  if (i < 0 || i >= m0) { a = 0; q = i; m = m0; }
  else if (j < 0 || j >= m1) { a = 1; q = j; m = m1; }
  else if (k < 0 || k >= m2) { a = 2; q = k; m = m2; }
  else return uc[fidx(g, c, i, j, k)];
  side = q < 0 ? 0 : 1;
  int kind = bc_of(g, a, side);
  int kk = side ? q - (m - 1) : -q;          // 1 or 2
  int qb;
  double sign = 1.0, base = 0.0;
  if (a == c) {
    int qe = side ? m - 1 : 0;
    double ub = uc[fidx(g, c, a == 0 ? qe : i, a == 1 ? qe : j, a == 2 ? qe : k)];
    if (kind == BC_OPEN) return ub;
    qb = side ? m - 1 - kk : kk;
    base = 2.0 * ub;
    sign = -1.0;
  } else {
    if (kind == BC_OPEN) qb = side ? m - 1 : 0;
    else qb = side ? m - kk : kk - 1;
    sign = (kind == BC_OPEN || kind == BC_AXIS) ? 1.0 : -1.0;
  }
  double v = uc[fidx(g, c, a == 0 ? qb : i, a == 1 ? qb : j, a == 2 ? qb : k)];
  return base + sign * v;
}

// clamp a cell index into the domain (zero-gradient access)
__device__ __forceinline__ double cellc(const Geo& g, const double* f, int i, int j, int k) {
  i = i < 0 ? 0 : (i >= g.n[0] ? g.n[0] - 1 : i);
  j = j < 0 ? 0 : (j >= g.n[1] ? g.n[1] - 1 : j);
  k = k < 0 ? 0 : (k >= g.n[2] ? g.n[2] - 1 : k);
  return f[cidx(g, i, j, k)];
}

// ------------------------------------------------------------------ FP64 <-> FP32 on the integer pipe
// On GB300 the hardware conversions issue on the FP64 pipe (about two per SM clock), so
// the mixed-precision kernels convert with integer operations instead.  Binary64 to
// binary32, round to nearest even (IEEE 754), written out for results in the normal
// binary32 range; zeros keep their sign; every other input (results that would be
// subnormal or overflow, infinities, NaN) takes the hardware conversion.
__device__ __forceinline__ float f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned e = (hi >> 20) & 0x7FFu;                       // biased binary64 exponent
  if (e - 897u <= 253u) {                                       // binary32 exponent 1 .. 254
    unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);           // leading 23 fraction bits
    const unsigned rest = lo & 0x1FFFFFFFu, half = 0x10000000u;  // the 29 dropped bits
    m += (rest > half) | ((rest == half) & (m & 1u));           // ties to even
    return __uint_as_float((hi & 0x80000000u) | (((e - 896u) << 23) + m));   // a carry bumps the exponent
  }
  if ((b << 1) == 0ull) return __uint_as_float(hi & 0x80000000u);
  return (float)x;
}
// binary32 to binary64 (exact) for normal numbers and zeros
__device__ __forceinline__ double f64_of(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
  if (e - 1u < 254u)
    return __longlong_as_double((long long)(s | ((unsigned long long)(e + 896u) << 52) |
                                            ((unsigned long long)(u & 0x7FFFFFu) << 29)));
  if ((u << 1) == 0u) return __longlong_as_double((long long)s);
  return (double)x;
}

// 1 / x in binary64 without the division sequence (GB300 retires about two binary64
// operations per SM clock, and a division takes a dozen): the binary32 reciprocal of x,
// rounded to nearest, as the seed of the Newton-Raphson iteration for f(y) = 1/y - x,
// y <- y + y (1 - x y) (each step squares the relative error: 2^-24, 2^-48, then below
// binary64 rounding; the result lies within one ulp of the correctly rounded 1 / x).
// Outside binary32's normal range (zero, subnormal, huge, inf, NaN) it divides.
__device__ __forceinline__ double rcp64(double x) {
  const float xf = f32_rn(x);
  const float ax = fabsf(xf);
  if (!(ax >= 1.5e-38f && ax <= 1.5e38f)) return 1.0 / x;
  double y = f64_of(__frcp_rn(xf));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// Minimum and maximum of binary64 values on the integer pipe (GB300's binary64 pipe
// also executes the comparisons and min/max): the IEEE 754 encodings, with the
// magnitude bits of negative values flipped, order as signed 64-bit integers exactly
// as the values do (-0 below +0), so the results equal fmin / fmax bit for bit for
// every non-NaN operand.
__device__ __forceinline__ long long ord64(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}
__device__ __forceinline__ double imax64(double a, double b) { return ord64(a) >= ord64(b) ? a : b; }
__device__ __forceinline__ double imin64(double a, double b) { return ord64(a) <= ord64(b) ? a : b; }
// clamp to [0, 1]
__device__ __forceinline__ double iclamp01(double a) { return imin64(1.0, imax64(0.0, a)); }
// a >= b, the same way (non-NaN operands)
__device__ __forceinline__ bool ige64(double a, double b) { return ord64(a) >= ord64(b); }

// ------------------------------------------------------------------ small formulas
// minmod(x, y): the operand of smaller magnitude when x and y are non-zero with the same
// sign, else 0 -- decided on the integer pipe (sign bits equal, magnitudes compared as
// unsigned encodings), with no binary64 instruction.  The same operand as the form
// x y > 0 ? sign(x) min(|x|, |y|) : 0 for every pair whose product does not underflow
// below the smallest subnormal (there the product test gives 0).
__device__ __forceinline__ double minmod(double x, double y) {
  const long long bx = __double_as_longlong(x), by = __double_as_longlong(y);
  const long long ax = bx & 0x7FFFFFFFFFFFFFFFLL, ay = by & 0x7FFFFFFFFFFFFFFFLL;
  const bool same = (bx ^ by) >= 0 && ax != 0 && ay != 0;
  return same ? (ax <= ay ? x : y) : 0.0;
}
// x and y the same pure phase value: both encodings that of +0 or both that of 1
__device__ __forceinline__ bool pure_pair(double x, double y) {
  const long long bx = __double_as_longlong(x);
  return bx == __double_as_longlong(y) && (bx == 0 || bx == 0x3FF0000000000000LL);
}
__device__ __forceinline__ double lim_up(double uu, double u, double d) { return u + 0.5 * minmod(u - uu, d - u); }
__device__ __forceinline__ double van_leer(double uu, double u, double d) {
  double dU = u - uu, dD = d - u, pr = dU * dD;
  return u + (pr > 0.0 ? pr * rcp64(dU + dD) : 0.0);
}

// ------------------------------------------------------------------ thermodynamics
__device__ __forceinline__ double psat(const Phys& p, double T) {
  return P_ATM * exp(p.cc_LMR * (p.iTb - rcp64(T)));
}
__device__ __forceinline__ double Y_from_y(const Phys& p, double y) {
  return y * p.M_l / (y * p.M_l + (1.0 - y) * p.M_g);
}
__device__ __forceinline__ double y_from_Y(const Phys& p, double Y) {
  const double m = Y * p.iM_l;
  return m * rcp64(m + (1.0 - Y) * p.iM_g);
}

// Peng-Robinson pure-component alpha factor sqrt(alpha(T)) = 1 + kappa (1 - sqrt(T / Tc))
// of component s, from sqrt(T) (shared by both components) and sqrt(1 / Tc); a(T) = a_c sq^2
// (the constants come from the host, Phys::pr_*)
__device__ __forceinline__ double pr_sq(const Phys& p, int s, double sqrtT) {
  return 1.0 + p.pr_k[s] * (1.0 - sqrtT * p.pr_siTc[s]);
}

// van der Waals mixing of the binary at fuel mole fraction y; A, B of the cubic
__device__ __forceinline__ void pr_mix_AB(const Phys& p, double T, double P, double y, double& A, double& B,
                                          double& a0, double& a01, double& am, double& bm) {
  const double sT = sqrt(T);
  const double s0 = pr_sq(p, 0, sT), s1 = pr_sq(p, 1, sT);
  a0 = p.pr_ac[0] * s0 * s0;
  const double a1 = p.pr_ac[1] * s1 * s1;
  a01 = p.pr_sqac01 * fabs(s0 * s1);          // sqrt(a0 a1) (1 - k_ij)
  const double y1 = 1.0 - y;
  am = y * y * a0 + y * y1 * a01 + y1 * y * a01 + y1 * y1 * a1;
  bm = y * p.pr_b[0] + y1 * p.pr_b[1];
  const double iRT = rcp64(R_GAS * T);
  A = am * P * iRT * iRT;
  B = bm * P * iRT;
}

// largest real root of z^3 + c2 z^2 + c1 z + c0 (Cardano; trigonometric form for three real roots)
__device__ inline double cubic_largest(double c2, double c1, double c0) {
  constexpr double third = 1.0 / 3.0, twentyseventh = 1.0 / 27.0;
  double p = c1 - c2 * c2 * third;
  double q = 2.0 * c2 * c2 * c2 * twentyseventh - c2 * c1 * third + c0;
  double disc = 0.25 * q * q + p * p * p * twentyseventh;
  double t;
  if (disc > 0.0) {
    double h = -0.5 * q;
    double w = h + copysign(sqrt(disc), h);
    double u = copysign(cbrt(fabs(w)), w);
    t = (u != 0.0) ? u - p / (3.0 * u) : 0.0;
  } else if (p == 0.0) {
    t = 0.0;
  } else {
    double m = 2.0 * sqrt(-p * third);
    double arg = 3.0 * q / (p * m);
    arg = fmin(1.0, fmax(-1.0, arg));
    t = m * cos(acos(arg) * third);
  }
  return t - c2 * third;
}

// The same root, refined instead of formed in binary64: Cardano's formula in binary32
// gives an estimate z0 within a few binary32 ulps of a well-separated largest root; a
// fixed-slope Newton iteration z <- z - f(z) / f'(z0) in binary64 (f evaluated in
// binary64, the slope rounded to binary32) contracts the error by about
// |f'(z0) - f'(z*)| / f'(z*) per step, which three steps take to rounding level.  The
// binary64 formula is used instead where the estimate is not clearly at a simple root
// (f'(z0) not well above zero: near a double root, where the contraction fails) or the
// last step still moved the root by more than 1e-8 relative.
__device__ inline double cubic_largest_refined(double c2, double c1, double c0) {
  const float a2 = f32_rn(c2), a1 = f32_rn(c1), a0 = f32_rn(c0);
  constexpr float third = 1.f / 3.f, twentyseventh = 1.f / 27.f;
  const float pp = a1 - a2 * a2 * third;
  const float qq = 2.f * a2 * a2 * a2 * twentyseventh - a2 * a1 * third + a0;
  const float disc = 0.25f * qq * qq + pp * pp * pp * twentyseventh;
  float t;
  if (disc > 0.f) {
    const float h = -0.5f * qq;
    const float w = h + copysignf(sqrtf(disc), h);
    const float u = copysignf(cbrtf(fabsf(w)), w);
    t = (u != 0.f) ? u - pp / (3.f * u) : 0.f;
  } else if (pp == 0.f) {
    t = 0.f;
  } else {
    const float m = 2.f * sqrtf(-pp * third);
    const float arg = fminf(1.f, fmaxf(-1.f, 3.f * qq / (pp * m)));
    t = m * cosf(acosf(arg) * third);
  }
  const float z0 = t - a2 * third;
  const float fp = (3.f * z0 + 2.f * a2) * z0 + a1;
  const float scale = 3.f * z0 * z0 + fabsf(2.f * a2 * z0) + fabsf(a1);
  if (!(fp > 1e-3f * scale)) return cubic_largest(c2, c1, c0);
  const double r = f64_of(1.f / fp);
  double z = f64_of(z0), dz = 0.0;
#pragma unroll
  for (int it = 0; it < 3; ++it) {
    dz = (((z + c2) * z + c1) * z + c0) * r;
    z -= dz;
  }
  if (!(fabs(dz) <= 1e-8 * fabs(z))) return cubic_largest(c2, c1, c0);
  return z;
}

// binary (fuel, inert) Peng-Robinson compressibility alone (the vapour root), for the
// gas density: pr_binary's cubic, its root refined (cubic_largest_refined)
__device__ inline double pr_binary_Z(const Phys& p, double T, double P, double y) {
  double A, B, a0, a01, am, bm;
  pr_mix_AB(p, T, P, y, A, B, a0, a01, am, bm);
  return cubic_largest_refined(-(1.0 - B), A - 3.0 * B * B - 2.0 * B, -(A * B - B * B - B * B * B));
}

// binary (fuel, inert) Peng-Robinson: vapour Z and ln phi_hat of the fuel at mole fraction y
__device__ inline void pr_binary(const Phys& p, double T, double P, double y, double& Z, double& lnphi0) {
  double A, B, a0, a01, am, bm;
  pr_mix_AB(p, T, P, y, A, B, a0, a01, am, bm);
  Z = cubic_largest(-(1.0 - B), A - 3.0 * B * B - 2.0 * B, -(A * B - B * B - B * B * B));
  const double s2 = 1.4142135623730951;
  const double b0 = p.pr_b[0];
  double logterm = log((Z + (1.0 + s2) * B) / (Z + (1.0 - s2) * B));
  double sa = y * a0 + (1.0 - y) * a01;
  lnphi0 = b0 / bm * (Z - 1.0) - log(Z - B) - A / (2.0 * s2 * B) * (2.0 * sa / am - b0 / bm) * logterm;
}

// liquid density at temperature T, linear through rho_l at the initial liquid temperature
// (Sec. 2.7 takes rho_L from correlations in T): rho_l + drl (T - T_drop), product and sum
// rounded separately; exactly rho_l for a constant density
__device__ __forceinline__ double rho_liq(const Phys& p, double T) {
  return __dadd_rn(p.rho_l, __dmul_rn(p.drl, T - p.T_drop));
}

// saturation mole fraction (Raoult, or the Peng-Robinson fixed point with the Poynting factor).
// y_start > 0 starts the fixed point there instead of at the Raoult value (a pinned cell's
// previous saturation value: the iteration then stops after a few steps at the same
// fixed point, within its 1e-13 tolerance).
__device__ inline double y_eq(const Phys& p, double T, unsigned* boil, double y_start = -1.0) {
  double p0 = psat(p, T);
  double y = p0 / p.P;
  if (y > Y_CLAMP) { y = Y_CLAMP; if (boil) *boil = 1u; }
  if (p.eq_model == 0) return y;
  if (y_start > 0.0 && y_start < Y_CLAMP) y = y_start;
  double Zp, lp;
  pr_binary(p, T, p0, 1.0, Zp, lp);
  double vL = p.M_l / rho_liq(p, T);
  double num = p0 * exp(lp) * exp(vL * (p.P - p0) / (R_GAS * T));
  for (int it = 0; it < 50; ++it) {
    double Z, l0;
    pr_binary(p, T, p.P, y, Z, l0);
    double yn = num / (p.P * exp(l0));
    if (yn > Y_CLAMP) { yn = Y_CLAMP; if (boil) *boil = 1u; }
    double dy = fabs(yn - y);
    y = yn;
    if (dy < 1e-13) break;
  }
  return y;
}

__device__ __forceinline__ double Y_eq(const Phys& p, double T, unsigned* boil, double Y_start = -1.0) {
  return Y_from_y(p, y_eq(p, T, boil, Y_start > 0.0 ? y_from_Y(p, Y_start) : -1.0));
}

__device__ inline double rho_gas(const Phys& p, double T, double Y) {
  if (p.const_props) return p.rhoG_const;
  double inv_m = Y * p.iM_l + (1.0 - Y) * p.iM_g;
  double Z = 1.0;
  if (p.eq_model != 0) Z = pr_binary_Z(p, T, p.P, y_from_Y(p, Y));
  return p.P * rcp64(Z * R_GAS * T * inv_m);
}

// ------------------------------------------------------------------ reductions
// Block-level sums of NV values, written to partials[v * gridDim.x + blockIdx.x].
// GB300 retires about two FP64 operations per SM clock, so the values are transposed
// through shared memory and value q is summed by warp q alone (blockDim.x / 32 adds
// per lane and a five-step shuffle), instead of a shuffle tree in every warp.  Fixed
// order: deterministic.  Blocks of at most TPB threads.
template <int NV>
__device__ inline void block_sum_store(double (&v)[NV], double* partials) {
  __shared__ double sh[NV][TPB];
#pragma unroll
  for (int q = 0; q < NV; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  for (int q = w; q < NV; q += nw) {
    double t = 0.0;
    for (int u = 0; u < nw; ++u) t += sh[q][lane + 32 * u];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) partials[q * gridDim.x + blockIdx.x] = t;
  }
}

template <int NV>
__device__ inline void block_max_store(double (&v)[NV], double* partials) {
  __shared__ double sh[NV][TPB];
#pragma unroll
  for (int q = 0; q < NV; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  for (int q = w; q < NV; q += nw) {
    double t = -1e300;
    for (int u = 0; u < nw; ++u) t = fmax(t, sh[q][lane + 32 * u]);
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_down_sync(0xffffffffu, t, o));
    if (lane == 0) partials[q * gridDim.x + blockIdx.x] = t;
  }
}

// Single-block sums (MAX = false) or maxima (MAX = true) of NV values from nblk
// partials each (partials[q * nblk + b]): all loads issue together, each value is
// finished by one warp through shared memory.  Result in thread 0.  Deterministic.
template <int NV, bool MAX>
__device__ inline void block_reduce_partials(const double* part, int nblk, double (&out)[NV]) {
  __shared__ double sh[NV][TPB];
  double t[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) t[q] = MAX ? -1e300 : 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const double x = __ldcg(part + q * nblk + b);
      t[q] = MAX ? fmax(t[q], x) : t[q] + x;
    }
#pragma unroll
  for (int q = 0; q < NV; ++q) sh[q][threadIdx.x] = t[q];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  for (int q = w; q < NV; q += nw) {
    double r = MAX ? -1e300 : 0.0;
    for (int u = 0; u < nw; ++u) r = MAX ? fmax(r, sh[q][lane + 32 * u]) : r + sh[q][lane + 32 * u];
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_down_sync(0xffffffffu, r, o);
      r = MAX ? fmax(r, y) : r + y;
    }
    __syncwarp();
    if (lane == 0) sh[q][0] = r;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) out[q] = sh[q][0];
  __syncthreads();
}

// Single-block sum of nblk partials per value (fixed order: deterministic).
__device__ inline double block_sum_partials(const double* part, int nblk) {
  __shared__ double sh[TPB / 32];
  double t = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) t += __ldcg(part + b);
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = t;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) r += sh[q];
  return r;   // valid in thread 0
}
__device__ inline double block_max_partials(const double* part, int nblk) {
  __shared__ double sh[TPB / 32];
  double t = -1e300;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) t = fmax(t, __ldcg(part + b));
  for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_down_sync(0xffffffffu, t, o));
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = t;
  __syncthreads();
  double r = -1e300;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) r = fmax(r, sh[q]);
  return r;
}

// True in the last block of the grid to reach this point (threadfence + atomic
// ticket; no waiting).  The block that gets the last ticket sees every other
// block's partials and resets the counter for the next launch.
__device__ __forceinline__ bool last_block(unsigned* cnt) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = atomicAdd(cnt, 1u) == gridDim.x - 1;
  __syncthreads();
  return am_last;
}

// grid of a reduction kernel with at most cap blocks (cap <= RED_BLOCKS, the partial buffers' size)
inline int red_grid_cap(long long n, int cap) {
  long long b = (n + TPB - 1) / TPB;
  if (cap < 1 || cap > RED_BLOCKS) cap = RED_BLOCKS;
  return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

inline int red_grid(long long n) {
  long long b = (n + TPB - 1) / TPB;
  return (int)(b < RED_BLOCKS ? (b < 1 ? 1 : b) : RED_BLOCKS);
}
inline int lin_grid(long long n) { return (int)((n + TPB - 1) / TPB); }

}  // namespace dg
