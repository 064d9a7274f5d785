// Kernels of one segregated time step (Sec. 3.1, Fig. Scheme):
// initial state, thermodynamics, evaporation flux, alpha source, alpha
// advection, mixture properties, assembly of the energy / species /
// momentum / pressure systems, velocity correction and diagnostics.
// One thread per cell or face; FP64 throughout.
#include "common.cuh"
#include "kernels.h"

namespace dg {

// ============================================================== initial state
// alpha: fraction of S^d sub-cell samples inside the sphere (S = 16 in 2D, 8 in 3D),
// computed without contracted multiply-adds so that every sample decision is exact.
__global__ void k_init(Geo g, Phys p, double* alpha, double* T, double* omega, double* rhoG) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  int i, j, k;
  decomp(id, g.n[0], g.n[1], i, j, k);
  int ci[3] = {i, j, k};
  const int S = g.axisym ? 16 : 8;
  double R2 = __dmul_rn(0.5 * p.D0, 0.5 * p.D0);
  // squared offsets of the sample coordinates per axis
  double d2a[3][16];
  int na = nact(g);
  for (int a = 0; a < na; ++a)
    for (int m = 0; m < S; ++m) {
      double frac = (m + 0.5) / S;
      double pos = __dmul_rn(__dadd_rn((double)ci[a], frac), g.h[a]);
      double dx = __dadd_rn(pos, -p.xc[a]);
      d2a[a][m] = __dmul_rn(dx, dx);
    }
  int count = 0;
  if (na == 2) {
    for (int m0 = 0; m0 < S; ++m0)
      for (int m1 = 0; m1 < S; ++m1) count += (__dadd_rn(d2a[0][m0], d2a[1][m1]) <= R2);
  } else {
    // quick classification of cells far from the sphere surface
    double lo = 0.0, hi = 0.0;
    for (int a = 0; a < 3; ++a) {
      double mn = d2a[a][0], mx = d2a[a][0];
      for (int m = 1; m < S; ++m) { mn = fmin(mn, d2a[a][m]); mx = fmax(mx, d2a[a][m]); }
      lo += mn; hi += mx;
    }
    if (lo > R2 * (1.0 + 1e-12)) count = 0;
    else if (hi < R2 * (1.0 - 1e-12)) count = S * S * S;
    else
      for (int m0 = 0; m0 < S; ++m0)
        for (int m1 = 0; m1 < S; ++m1) {
          double s01 = __dadd_rn(d2a[0][m0], d2a[1][m1]);
          for (int m2 = 0; m2 < S; ++m2) count += (__dadd_rn(s01, d2a[2][m2]) <= R2);
        }
  }
  double a = (double)count / (double)(na == 2 ? S * S : S * S * S);
  alpha[id] = a;
  // distance of the cell centre to the droplet centre
  double d2 = 0.0;
  for (int q = 0; q < na; ++q) {
    double x = (ci[q] + 0.5) * g.h[q] - p.xc[q];
    d2 = d2 + x * x;
  }
  double r = sqrt(d2);
  double rs = 0.5 * p.D0;
  double t;
  if (p.const_props) {
    t = p.T_drop;
  } else {
    double Rf = 2.0 * p.D0;
    double w = (1.0 / fmax(r, rs) - 1.0 / Rf) / (1.0 / rs - 1.0 / Rf);
    w = fmin(1.0, fmax(0.0, w));
    t = p.T_amb + (p.T_drop - p.T_amb) * w;
  }
  if (p.T_perturb != 0.0) {
    // SplitMix64 (Steele, Lea & Flood 2014) of seed xor the linear cell index
    unsigned long long z = (p.seed ^ (unsigned long long)id) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    double u = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
    t = t * (1.0 + p.T_perturb * u);
  }
  T[id] = t;
  double Ys = Y_eq(p, p.T_drop, nullptr);
  double w;
  if (a >= 0.5) {
    w = Y_eq(p, t, nullptr);
  } else {
    double Rinf = p.const_props ? 4e-3 : 2.0 * p.D0;
    double ww = (1.0 / fmax(r, rs) - 1.0 / Rinf) / (1.0 / rs - 1.0 / Rinf);
    ww = fmin(1.0, fmax(0.0, ww));
    w = 1.0 - exp(log(1.0 - Ys) * ww);
    if (r >= Rinf) w = 0.0;
  }
  if (solid_cell(g, id)) {   // the fibre: no liquid, the liquid's initial temperature, no vapour
    alpha[id] = 0.0;
    t = p.T_drop;
    T[id] = t;
    w = 0.0;
  }
  omega[id] = w;
  rhoG[id] = rho_gas(p, t, w);
}

// centripetal potential xi = xi0 D_f / (2 max(r, D_f)) at the cell centres (Eq. magneticpotential);
// static, computed once
__global__ void k_xi(Geo g, Phys p, double* xi) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  int q[3];
  decomp(id, g.n[0], g.n[1], q[0], q[1], q[2]);
  int na = nact(g);
  double d2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    if (a >= na) break;
    double x = (q[a] + 0.5) * g.h[a] - p.xc[a];
    d2 = d2 + x * x;
  }
  xi[id] = p.xi0 * p.Df / (2.0 * fmax(sqrt(d2), p.Df));
}

// ============================================================== S0 thermodynamics
// Saturation value written into the liquid (alpha >= 1/2), gas density at T^n.
// The state rho_G left by the previous step is rho_gas(T, omega) of the same T and
// omega (and the pinned values Y_eq(T) are unchanged), so only liquid cells are
// re-evaluated, unless a field was overwritten since (*dirty != 0).
// (also resets the step's solver statistics, scal[SC_ITS_P .. SC_RES_P])
__global__ void k_thermo_pin(Geo g, Phys p, const double* alpha, const double* T, double* omega,
                             const double* rhoG, double* rhoG_old, unsigned* flags, const int* dirty, double* scal) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  if (id <= SC_RES_P - SC_ITS_P) scal[SC_ITS_P + id] = 0.0;
  unsigned boil = 0;
  double w = omega[id];
  bool liq = alpha[id] >= 0.5;
  if (liq) { w = Y_eq(p, T[id], &boil, w); omega[id] = w; }
  rhoG_old[id] = (liq || *dirty) ? rho_gas(p, T[id], w) : rhoG[id];
  if (boil) atomicOr(flags, (unsigned)DROPLET_FLAG_BOILING);
}

// the six neighbour values of a central difference at (i, j, k) with those inside the fibre
// replaced by the cell's own value (zero gradient across the sphere)
__device__ __forceinline__ void fibre_mask6(const Geo& g, const double* f, int i, int j, int k, double& e, double& w,
                                            double& n, double& s, double& t, double& b) {
  const double own = f[cidx(g, i, j, k)];
  if (solid_nb(g, i + 1, j, k)) e = own;
  if (solid_nb(g, i - 1, j, k)) w = own;
  if (solid_nb(g, i, j + 1, k)) n = own;
  if (solid_nb(g, i, j - 1, k)) s = own;
  if (g.act3) {
    if (solid_nb(g, i, j, k + 1)) t = own;
    if (solid_nb(g, i, j, k - 1)) b = own;
  }
}

// central gradient of alpha at cell (i,j,k) with the alpha ghost rule
// (a neighbour inside the fibre takes the cell's own value: zero gradient across the sphere)
__device__ __forceinline__ void grad_alpha(const Geo& g, const double* al, int i, int j, int k, double gr[3]) {
  double e = cellg(g, al, i + 1, j, k, R_ALPHA, 0, 0, 0, 0), w = cellg(g, al, i - 1, j, k, R_ALPHA, 0, 0, 0, 0);
  double n = cellg(g, al, i, j + 1, k, R_ALPHA, 0, 0, 0, 0), s = cellg(g, al, i, j - 1, k, R_ALPHA, 0, 0, 0, 0);
  double t = g.act3 ? cellg(g, al, i, j, k + 1, R_ALPHA, 0, 0, 0, 0) : 0.0;
  double b = g.act3 ? cellg(g, al, i, j, k - 1, R_ALPHA, 0, 0, 0, 0) : 0.0;
  if (g.fib) fibre_mask6(g, al, i, j, k, e, w, n, s, t, b);
  gr[0] = (e - w) * (0.5 * g.ih[0]);
  gr[1] = (n - s) * (0.5 * g.ih[1]);
  gr[2] = g.act3 ? (t - b) * (0.5 * g.ih[2]) : 0.0;
}
// grad_alpha, and whether it vanishes identically: equal neighbours on every axis
// (compared as encodings, on the integer pipe) give exactly +0 differences, so such a
// flat cell can skip the binary64 arithmetic that depends on the gradient
__device__ __forceinline__ bool grad_alpha_flat(const Geo& g, const double* al, int i, int j, int k, double gr[3]) {
  const double e0 = cellg(g, al, i + 1, j, k, R_ALPHA, 0, 0, 0, 0), w0 = cellg(g, al, i - 1, j, k, R_ALPHA, 0, 0, 0, 0);
  const double n0 = cellg(g, al, i, j + 1, k, R_ALPHA, 0, 0, 0, 0), s0 = cellg(g, al, i, j - 1, k, R_ALPHA, 0, 0, 0, 0);
  const double t0 = g.act3 ? cellg(g, al, i, j, k + 1, R_ALPHA, 0, 0, 0, 0) : 0.0;
  const double b0 = g.act3 ? cellg(g, al, i, j, k - 1, R_ALPHA, 0, 0, 0, 0) : 0.0;
  double e = e0, w = w0, n = n0, s = s0, t = t0, b = b0;
  if (g.fib) fibre_mask6(g, al, i, j, k, e, w, n, s, t, b);
  if (__double_as_longlong(e) == __double_as_longlong(w) && __double_as_longlong(n) == __double_as_longlong(s) &&
      __double_as_longlong(t) == __double_as_longlong(b)) {
    gr[0] = gr[1] = gr[2] = 0.0;
    return true;
  }
  gr[0] = (e - w) * (0.5 * g.ih[0]);
  gr[1] = (n - s) * (0.5 * g.ih[1]);
  gr[2] = g.act3 ? (t - b) * (0.5 * g.ih[2]) : 0.0;
  return false;
}
__device__ __forceinline__ double norm_rn(const double gr[3], int na) {
  double s = __dadd_rn(__dmul_rn(gr[0], gr[0]), __dmul_rn(gr[1], gr[1]));
  if (na == 3) s = __dadd_rn(s, __dmul_rn(gr[2], gr[2]));
  return sqrt(s);
}

// ============================================================== S1 evaporation flux
// Interface cells |grad alpha| > 1e-8/h_min; adjacent gas cell = first cell at
// distance s h_min (s = 1, 2, 3) along n = -grad(alpha)/|grad(alpha)| with
// alpha < 1e-3 (axis mirrored, stop at the domain edge); j = -rho D grad(omega)
// + rho omega v there; m_raw = -j . grad(alpha) (Eqs. massflux, globalFlux).
// Partial sums of m_raw V and f(alpha) m_raw V per block.
template <int NA>
__global__ void k_evap_raw(Geo g, Phys p, const double* alpha, const double* omega, const double* rhoG,
                           const double* T, const double* u0, const double* u1, const double* u2,
                           double* mraw, int* adj, double* partials, unsigned* flags) {
  double acc[2] = {0.0, 0.0};
  constexpr int na = NA;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < g.N; id += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    decomp(id, g.n[0], g.n[1], i, j, k);
    double gr[3];
    const bool flat = grad_alpha_flat(g, alpha, i, j, k, gr);
    const double gm = flat ? 0.0 : norm_rn(gr, na);
    double m = 0.0;
    int found = -1;
    if (gm > g.gthr && !solid_cell(g, id)) {   // (the fibre's cells are never interface cells)
      double nh[3] = {-gr[0] / gm, -gr[1] / gm, -gr[2] / gm};
      int ci[3] = {i, j, k};
      int q[3] = {0, 0, 0};
      for (int s = 1; s <= 3 && found < 0; ++s) {
        bool inside = true;
        #pragma unroll
        for (int a = 0; a < na; ++a) {
          double ratio = g.hmin * g.ih[a];
          double xi = __dadd_rn((double)ci[a] + 0.5, __dmul_rn(__dmul_rn((double)s, ratio), nh[a]));
          if (g.axisym && a == 0) xi = fabs(xi);
          double fq = floor(xi);
          if (fq < 0.0 || fq >= (double)g.n[a]) { inside = false; break; }
          q[a] = (int)fq;
        }
        if (!inside) break;
        if (!g.act3) q[2] = 0;
        long long qi = cidx(g, q[0], q[1], q[2]);
        if (solid_cell(g, qi)) continue;   // the march passes over the fibre's cells
        if (alpha[qi] < ALPHA_GAS) found = (int)qi;
      }
      if (found < 0) {
        atomicOr(flags, (unsigned)DROPLET_FLAG_ADJ_NOT_FOUND);
      } else {
        // total flux at the adjacent cell Q
        double aQ = alpha[found], rgQ = rhoG[found], wQ = omega[found];
        double rhoQ = aQ * (p.drl == 0.0 ? p.rho_l : rho_liq(p, T[found])) + (1.0 - aQ) * rgQ;
        double DQ = aQ * p.D_l + (1.0 - aQ) * p.D_gas;
        int qi, qj, qk;
        decomp(found, g.n[0], g.n[1], qi, qj, qk);
        double gw[3];
        double we = cellg(g, omega, qi + 1, qj, qk, R_TO, 0.0, u0, u1, u2), ww = cellg(g, omega, qi - 1, qj, qk, R_TO, 0.0, u0, u1, u2);
        double wn = cellg(g, omega, qi, qj + 1, qk, R_TO, 0.0, u0, u1, u2), ws = cellg(g, omega, qi, qj - 1, qk, R_TO, 0.0, u0, u1, u2);
        double wt = g.act3 ? cellg(g, omega, qi, qj, qk + 1, R_TO, 0.0, u0, u1, u2) : 0.0;
        double wb = g.act3 ? cellg(g, omega, qi, qj, qk - 1, R_TO, 0.0, u0, u1, u2) : 0.0;
        if (g.fib) fibre_mask6(g, omega, qi, qj, qk, we, ww, wn, ws, wt, wb);
        gw[0] = (we - ww) * (0.5 * g.ih[0]);
        gw[1] = (wn - ws) * (0.5 * g.ih[1]);
        gw[2] = g.act3 ? (wt - wb) * (0.5 * g.ih[2]) : 0.0;
        double vc[3];
        vc[0] = 0.5 * (u0[fidx(g, 0, qi, qj, qk)] + u0[fidx(g, 0, qi + 1, qj, qk)]);
        vc[1] = 0.5 * (u1[fidx(g, 1, qi, qj, qk)] + u1[fidx(g, 1, qi, qj + 1, qk)]);
        vc[2] = g.act3 ? 0.5 * (u2[fidx(g, 2, qi, qj, qk)] + u2[fidx(g, 2, qi, qj, qk + 1)]) : 0.0;
        double s = 0.0;
        #pragma unroll
        for (int a = 0; a < na; ++a) {
          double ja = -rhoQ * DQ * gw[a] + rhoQ * wQ * vc[a];
          s = s + ja * gr[a];
        }
        m = -s;
      }
    }
    mraw[id] = m;
    adj[id] = found;
    if (m != 0.0) {   // (a zero m adds zeros: alpha is in [0, 1], the root finite)
      double V = cellV(g, i);
      double a = alpha[id];
      acc[0] += m * V;
      acc[1] += sqrt(a * (1.0 - a)) * m * V;
    }
  }
  block_sum_store<2>(acc, partials);
}

// K = sum(m_raw V) / sum(f m_raw V) (Eq. alphafunction normalisation)
__global__ void k_evap_K(const double* partials, int nblk, double* scal, unsigned* flags) {
  double s1 = block_sum_partials(partials, nblk);
  double s2 = block_sum_partials(partials + nblk, nblk);
  if (threadIdx.x == 0) {
    if (fabs(s2) < 1e-300) { scal[SC_K] = 0.0; atomicOr(flags, (unsigned)DROPLET_FLAG_NO_INTERFACE); }
    else scal[SC_K] = s1 / s2;
  }
}

// ============================================================== S2 alpha source
// (also clears the state-overwritten flag that S0 consumed)
// (alpha_star_f, when given: alpha* rounded to binary32 for the mixed-precision face
// stencils.)  Cells without a raw flux (all but the interface band) keep alpha* = alpha
// and m = 0 without the binary64 square root, cap and update, whose results there are
// exactly those values.
__global__ void k_alpha_source(Geo g, Phys p, const double* alpha, const double* mraw, const double* scal,
                               const double* T, const double* expand, double* mdot, double* alpha_star,
                               float* alpha_star_f, unsigned* flags, int* dirty) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  if (id == 0) *dirty = 0;
  const double a = alpha[id];
  const double mr = mraw[id];
  double m = 0.0, as = a;
  if ((__double_as_longlong(mr) << 1) != 0) {      // mraw != 0, tested on the integer pipe
    const double K = scal[SC_K];
    m = (K == 0.0) ? 0.0 : K * sqrt(a * (1.0 - a)) * mr;
    const double rl = p.drl == 0.0 ? p.rho_l : rho_liq(p, T[id]);
    const double cap = rl * a * idt_of(p);
    if (m > cap) { m = cap; atomicOr(flags, (unsigned)DROPLET_FLAG_MDOT_CAPPED); }
    as = p.drl == 0.0 ? a - dt_of(p) * m * p.irho_l : a - dt_of(p) * m / rl;
  }
  if (expand) as = as - dt_of(p) * expand[id];
  mdot[id] = m;
  alpha_star[id] = as;
  if (alpha_star_f) alpha_star_f[id] = f32_rn(as);
}

// ============================================================== S3 alpha advection (FCT)
// Per face of direction a: low-order flux FL = phi alpha_upwind and the
// antidiffusive flux AF = FH - FL (interior faces only), FH = phi alpha_vanLeer
// + C_alpha |phi| (n_f . e_a) a_c (1 - a_c).
template <int DIR, int NA>
__global__ void k_adv_faces(Geo g, Phys p, const double* as, const double* ua, double* FL, double* AF) {
  constexpr int a = DIR;
  long long nf = nfaces(g, a);
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= nf) return;
  int m0 = g.n[0] + (a == 0), m1 = g.n[1] + (a == 1);
  int f[3];
  decomp(id, m0, m1, f[0], f[1], f[2]);
  int L[3] = {f[0], f[1], f[2]}, R[3] = {f[0], f[1], f[2]};
  L[a] -= 1;
  double phi = ua[id] * faceA(g, a, f[0]) * dt_of(p);
  double aL = cellg(g, as, L[0], L[1], L[2], R_ALPHA, 0, 0, 0, 0);
  double aR = cellg(g, as, R[0], R[1], R[2], R_ALPHA, 0, 0, 0, 0);
  bool pos = phi >= 0.0;
  FL[id] = phi * (pos ? aL : aR);
  double A = 0.0;
  // a face between two cells of the same pure phase (alpha both 0 or both 1, compared as
  // encodings on the integer pipe) has FH = FL exactly: the van Leer increment vanishes
  // with the downwind difference and the compression term with a_c (1 - a_c); its
  // antidiffusive flux is +0 without the gradient arithmetic
  if (f[a] > 0 && f[a] < g.n[a] && !pure_pair(aL, aR)) {
    int LL[3] = {L[0], L[1], L[2]}, RR[3] = {R[0], R[1], R[2]};
    LL[a] -= 1;
    RR[a] += 1;
    double aLL = cellg(g, as, LL[0], LL[1], LL[2], R_ALPHA, 0, 0, 0, 0);
    double aRR = cellg(g, as, RR[0], RR[1], RR[2], R_ALPHA, 0, 0, 0, 0);
    double aVL = pos ? van_leer(aLL, aL, aR) : van_leer(aRR, aR, aL);
    double gL[3], gR[3];
    grad_alpha(g, as, L[0], L[1], L[2], gL);
    grad_alpha(g, as, R[0], R[1], R[2], gR);
    double gf[3] = {gL[0] + gR[0], gL[1] + gR[1], gL[2] + gR[2]};
    double gfm = sqrt(gf[0] * gf[0] + gf[1] * gf[1] + (g.act3 ? gf[2] * gf[2] : 0.0));
    double ne = gfm > g.gthr ? gf[a] / gfm : 0.0;
    double ac = 0.5 * (aL + aR);
    double FH = phi * aVL + p.C_alpha * fabs(phi) * ne * ac * (1.0 - ac);
    A = FH - FL[id];
  }
  AF[id] = A;
}

__device__ __forceinline__ double face_net(const Geo& g, const double* F0, const double* F1, const double* F2,
                                           int i, int j, int k) {
  double s = F0[fidx(g, 0, i + 1, j, k)] - F0[fidx(g, 0, i, j, k)];
  s += F1[fidx(g, 1, i, j + 1, k)] - F1[fidx(g, 1, i, j, k)];
  if (g.act3) s += F2[fidx(g, 2, i, j, k + 1)] - F2[fidx(g, 2, i, j, k)];
  return s;
}

__global__ void k_adv_low(Geo g, const double* as, const double* F0, const double* F1, const double* F2, double* aL) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  int i, j, k;
  decomp(id, g.n[0], g.n[1], i, j, k);
  aL[id] = as[id] - face_net(g, F0, F1, F2, i, j, k) * rcp64(cellV(g, i));
}

// ============================================================== S4 mixture properties
__device__ __forceinline__ void props_cell(const Phys& p, long long id, double a, const double* rhoG,
                                           const double* omega, const double* T, double* rho, double* mu,
                                           double* kc, double* cp, double* D) {
  const double w = omega[id];
  const long long ba = __double_as_longlong(a);
  if (ba == 0) {                          // pure gas: the mixture rule gives the gas values exactly
    rho[id] = rhoG[id];
    mu[id] = p.mu_g;
    kc[id] = p.k_g;
    cp[id] = w * p.cp_v + (1.0 - w) * p.cp_g;
    D[id] = p.D_gas;
    return;
  }
  if (ba == 0x3FF0000000000000LL) {       // pure liquid (alpha = 1)
    rho[id] = p.drl == 0.0 ? p.rho_l : rho_liq(p, T[id]);
    mu[id] = p.mu_l;
    kc[id] = p.k_l;
    cp[id] = p.cp_l;
    D[id] = p.D_l;
    return;
  }
  rho[id] = a * (p.drl == 0.0 ? p.rho_l : rho_liq(p, T[id])) + (1.0 - a) * rhoG[id];
  mu[id] = a * p.mu_l + (1.0 - a) * p.mu_g;
  kc[id] = a * p.k_l + (1.0 - a) * p.k_g;
  double cpG = w * p.cp_v + (1.0 - w) * p.cp_g;
  cp[id] = a * p.cp_l + (1.0 - a) * cpG;
  D[id] = a * p.D_l + (1.0 - a) * p.D_gas;
}

// props_cell into the PropsOut arrays, and their binary32 copies when asked for; the fibre's
// cells conduct and diffuse nothing (no flux of T or omega across the sphere)
__device__ __forceinline__ void props_out(const Phys& p, long long id, double a, const PropsOut& po) {
  props_cell(p, id, a, po.rhoG, po.omega, po.T, po.rho, po.mu, po.kc, po.cp, po.D);
  if (po.solid && po.solid[id]) {
    po.kc[id] = 0.0;
    po.D[id] = 0.0;
  }
  if (po.s.T) {
    po.s.T[id] = f32_rn(po.T[id]);
    po.s.w[id] = f32_rn(po.omega[id]);
    po.s.k[id] = f32_rn(po.kc[id]);
    po.s.gD[id] = f32_rn(po.rho[id] * po.D[id]);
    po.s.mu[id] = f32_rn(po.mu[id]);
  }
}

__global__ void k_faces_f32(const double* u0, const double* u1, const double* u2, float* f0, float* f1, float* f2,
                            long long n0, long long n1, long long n2) {
  const long long n = n0 + n1 + n2;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n; id += (long long)gridDim.x * blockDim.x) {
    if (id < n0) f0[id] = f32_rn(u0[id]);
    else if (id < n0 + n1) f1[id - n0] = f32_rn(u1[id - n0]);
    else f2[id - n0 - n1] = f32_rn(u2[id - n0 - n1]);
  }
}

// Zalesak limiter ratios R+ and R- from the local bounds over the cell and its face neighbours.
template <int NA>
__global__ void k_adv_limit(Geo g, const double* as, const double* aL, const double* A0, const double* A1,
                            const double* A2, double* Rp, double* Rm) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  int i, j, k;
  decomp(id, g.n[0], g.n[1], i, j, k);
  constexpr int na = NA;
  const double* AA[3] = {A0, A1, A2};
  double Alo[3], Ahi[3];
  long long anyA = 0;   // OR of the encodings without sign: 0 when every face flux is +-0
  #pragma unroll
  for (int a = 0; a < na; ++a) {
    int hi[3] = {i, j, k};
    hi[a] += 1;
    Alo[a] = AA[a][fidx(g, a, i, j, k)];
    Ahi[a] = AA[a][fidx(g, a, hi[0], hi[1], hi[2])];
    anyA |= (__double_as_longlong(Alo[a]) | __double_as_longlong(Ahi[a])) << 1;
  }
  if (anyA == 0) {   // P+ = P- = 0: both ratios are 0
    Rp[id] = 0.0;
    Rm[id] = 0.0;
    return;
  }
  double amax = imax64(as[id], aL[id]), amin = imin64(as[id], aL[id]);
  #pragma unroll
  for (int a = 0; a < na; ++a)
    #pragma unroll
    for (int sh = -1; sh <= 1; sh += 2) {
      int q[3] = {i, j, k};
      q[a] += sh;
      if (q[a] < 0 || q[a] >= g.n[a]) continue;
      long long qi = cidx(g, q[0], q[1], q[2]);
      if (solid_cell(g, qi)) continue;   // nor do the fibre's cells
      const double sq = as[qi], lq = aL[qi];
      amax = imax64(amax, imax64(sq, lq));
      amin = imin64(amin, imin64(sq, lq));
    }
  amax = imin64(amax, 1.0);
  amin = imax64(amin, 0.0);
  double Pp = 0.0, Pm = 0.0;
  #pragma unroll
  for (int a = 0; a < na; ++a) {
    Pp += imax64(0.0, Alo[a]) + imax64(0.0, -Ahi[a]);
    Pm += imax64(0.0, -Alo[a]) + imax64(0.0, Ahi[a]);
  }
  double V = cellV(g, i);
  double Qp = (amax - aL[id]) * V, Qm = (aL[id] - amin) * V;
  // (Q = 0 gives 0 directly: Q / P for a subnormal P would be 0 x inf through the reciprocal)
  Rp[id] = Pp > 0.0 && Qp > 0.0 ? iclamp01(Qp * rcp64(Pp)) : 0.0;
  Rm[id] = Pm > 0.0 && Qm > 0.0 ? iclamp01(Qm * rcp64(Pm)) : 0.0;
}

__device__ __forceinline__ double limited_flux(const Geo& g, int a, const double* A, const double* Rp,
                                               const double* Rm, int f0, int f1, int f2) {
  double Af = A[fidx(g, a, f0, f1, f2)];
  if ((__double_as_longlong(Af) << 1) == 0) return 0.0;   // Af == +-0, on the integer pipe
  int L[3] = {f0, f1, f2};
  L[a] -= 1;
  long long li = cidx(g, L[0], L[1], L[2]), ri = cidx(g, f0, f1, f2);
  double C = Af >= 0.0 ? imin64(Rp[ri], Rm[li]) : imin64(Rp[li], Rm[ri]);
  return C * Af;
}

// alpha^{n+1} = alpha^L - sum C A / V, clipped to [0, 1] with the clipped volume summed.
template <int NA>
// (and the mixture properties of the cell from alpha^{n+1}, S4)
__global__ void k_adv_update(Geo g, Phys p, const double* aL, const double* A0, const double* A1, const double* A2,
                             const double* Rp, const double* Rm, double* alpha, double* partials, unsigned* flags,
                             PropsOut po) {
  double acc[2] = {0.0, 0.0};
  const double* AA[3] = {A0, A1, A2};
  constexpr int na = NA;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < g.N; id += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    decomp(id, g.n[0], g.n[1], i, j, k);
    double s = 0.0;
    #pragma unroll
    for (int a = 0; a < na; ++a) {
      int hi[3] = {i, j, k};
      hi[a] += 1;
      s += limited_flux(g, a, AA[a], Rp, Rm, hi[0], hi[1], hi[2]) - limited_flux(g, a, AA[a], Rp, Rm, i, j, k);
    }
    double V = cellV(g, i);
    // no limited flux (s = +-0): alpha^L itself, without the reciprocal (the clamp below
    // maps -0 to +0 either way)
    double an = ((__double_as_longlong(s) << 1) == 0) ? aL[id] : aL[id] - s * rcp64(V);
    double ac = iclamp01(an);
    if (ac != an) { acc[1] += 1.0; acc[0] += (an - ac) * V; }
    alpha[id] = ac;
    props_out(p, id, ac, po);
  }
  block_sum_store<2>(acc, partials);
}

// ============================================================== S3, geometric (reading R30)
// The paper moves the interface geometrically (Sec. 2.1, Eq. advection, isoAdvector).  On
// the uniform grid: one sweep per axis; in each, every partly filled cell holds a plane
// (PLIC) and a face passes the liquid of its donor's swept slab.  Geometry of a plane in
// the unit box [0, 1]^d, liquid side n . xi <= beta, normal in box coordinates (component a
// times h_a): the clipped volume by inclusion-exclusion over the box corners, arranged so
// that a vanishing component is only ever divided into a bounded ratio.

// fraction of the unit square below m1 x + m2 y = a (m1 <= m2, m1 + m2 = 1, 0 <= a <= 1/2)
__device__ __forceinline__ double geo_frac2(double m1, double m2, double a) {
  if (a <= m1) return m1 > 0.0 ? (a / m1) * a / (2.0 * m2) : 0.0;
  return (2.0 * a - m1) / (2.0 * m2);
}

// fraction of the unit cube below m . x = a (m1 <= m2 <= m3, sum 1, 0 <= a <= 1/2):
// 6 m1 m2 m3 V = a^3 - sum_i (a - m_i)_+^3, each corner term (a - m_i)^3 / m1 taken as
// (t / m1) t^2 with t <= m1; the slab beyond a = m1 + m2 when m3 >= m1 + m2 is linear
__device__ __forceinline__ double geo_frac3(double m1, double m2, double m3, double a) {
  if (a <= m1) return m1 > 0.0 ? (a / m1) * a * a / (6.0 * m2 * m3) : 0.0;
  if (a <= m2) return (a * a - a * m1 + m1 * m1 / 3.0) / (2.0 * m2 * m3);
  const double m12 = m1 + m2;
  if (m12 <= m3 && a > m12) return (2.0 * a - m12) / (2.0 * m3);
  const double t2 = fmax(a - m2, 0.0), t3 = fmax(a - m3, 0.0);
  const double r2 = m1 > 0.0 ? t2 / m1 : 0.0, r3 = m1 > 0.0 ? t3 / m1 : 0.0;
  return (3.0 * a * a - 3.0 * a * m1 + m1 * m1 - r2 * t2 * t2 - r3 * t3 * t3) / (6.0 * m2 * m3);
}

// |n| sorted ascending and scaled to unit sum; s = sum |n| (0: no plane)
__device__ __forceinline__ void geo_sorted(int d, double n0, double n1, double n2, double m[3], double& s) {
  double x = fabs(n0), y = fabs(n1), z = d == 3 ? fabs(n2) : 0.0;
  s = d == 3 ? (x + y) + z : x + y;
  const double ss = s > 0.0 ? s : 1.0;
  x = x / ss;
  y = y / ss;
  z = z / ss;
  if (d == 2) {
    m[0] = fmin(x, y);
    m[1] = fmax(x, y);
    m[2] = 0.0;
    return;
  }
  // three-element sorting network
  double t;
  if (x > y) { t = x; x = y; y = t; }
  if (y > z) { t = y; y = z; z = t; }
  if (x > y) { t = x; x = y; y = t; }
  m[0] = x;
  m[1] = y;
  m[2] = z;
}

// fraction of the unit box on the side n . xi <= beta
__device__ double geo_cut_fraction(int d, double n0, double n1, double n2, double beta) {
  const double neg = d == 3 ? (fmin(n0, 0.0) + fmin(n1, 0.0)) + fmin(n2, 0.0) : fmin(n0, 0.0) + fmin(n1, 0.0);
  beta -= neg;                          // reflect the axes with negative components
  double m[3], s;
  geo_sorted(d, n0, n1, n2, m, s);
  if (!(s > 0.0)) return beta >= 0.0 ? 1.0 : 0.0;
  const double a = beta / s;
  if (a <= 0.0) return 0.0;
  if (a >= 1.0) return 1.0;
  const bool hi = a > 0.5;
  const double b = fmin(fmax(hi ? 1.0 - a : a, 0.0), 0.5);
  const double v = d == 2 ? geo_frac2(m[0], m[1], b) : geo_frac3(m[0], m[1], m[2], b);
  return hi ? 1.0 - v : v;
}

// the plane constant beta that cuts the fraction f (0 < f < 1) from the unit box: closed
// forms on the square-root, cube-root, quadratic and linear pieces, bisection on the cubic
// pieces (60 halvings); 0 for a zero normal
__device__ double geo_plane_constant(int d, double n0, double n1, double n2, double f) {
  double m[3], s;
  geo_sorted(d, n0, n1, n2, m, s);
  if (!(s > 0.0)) return 0.0;
  const bool hi = f > 0.5;
  const double gv = hi ? 1.0 - f : f;
  const double m1 = m[0], m2 = m[1];
  double a;
  if (d == 2) {
    const double g1 = m1 > 0.0 ? m1 / (2.0 * m2) : 0.0;
    a = gv <= g1 ? sqrt(2.0 * m1 * m2 * gv) : gv * m2 + 0.5 * m1;
  } else {
    const double m3 = m[2], m12 = m1 + m2;
    if (gv <= geo_frac3(m1, m2, m3, m1)) {
      a = cbrt(6.0 * m1 * m2 * m3 * gv);
    } else if (gv <= geo_frac3(m1, m2, m3, m2)) {
      a = 0.5 * (m1 + sqrt(fmax(8.0 * m2 * m3 * gv - m1 * m1 / 3.0, 0.0)));
    } else if (m12 <= m3 && gv >= geo_frac3(m1, m2, m3, m12)) {
      a = gv * m3 + 0.5 * m12;
    } else {
      double lo = m2, up = m12 <= m3 ? m12 : 0.5;
      for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + up);
        if (geo_frac3(m1, m2, m3, mid) < gv) lo = mid;
        else up = mid;
      }
      a = 0.5 * (lo + up);
    }
  }
  if (hi) a = 1.0 - a;
  const double neg = d == 3 ? (fmin(n0, 0.0) + fmin(n1, 0.0)) + fmin(n2, 0.0) : fmin(n0, 0.0) + fmin(n1, 0.0);
  return a * s + neg;
}

// alpha of cell (i, j, k) for the reconstruction, clamped into [0, 1]: across the axis the
// mirror image, beyond every other boundary (and at a corner beyond two) 0
__device__ __forceinline__ double geo_alpha(const Geo& g, const double* a, int i, int j, int k) {
  const bool oi = i < 0 || i >= g.n[0], oj = j < 0 || j >= g.n[1], ok = k < 0 || k >= g.n[2];
  if (!oi && !oj && !ok) return iclamp01(a[cidx(g, i, j, k)]);
  if (oi && !oj && !ok && i == -1 && g.bc[0][0] == BC_AXIS) return iclamp01(a[cidx(g, 0, j, k)]);
  return 0.0;
}

// Plane of every partly filled cell of the sweep's input: Youngs' normal (minus the
// gradient, each difference along an axis summed over the neighbouring rows with weights
// (1, 2, 1) per other axis; box coordinates) and the constant that cuts the cell's alpha.
template <int NA>
__global__ void k_geo_plane(Geo g, const double* a, double* N0, double* N1, double* N2, double* B) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  int i, j, k;
  decomp(id, g.n[0], g.n[1], i, j, k);
  const double ac = iclamp01(a[id]);
  double n[3] = {0.0, 0.0, 0.0}, beta = 0.0;
  if (ac > 0.0 && ac < 1.0) {
    constexpr double w[3] = {1.0, 2.0, 1.0};
    #pragma unroll
    for (int ax = 0; ax < NA; ++ax) {
      double acc = 0.0;
      const int o1 = ax == 0 ? 1 : 0, o2 = NA == 3 ? (ax == 2 ? 1 : 2) : -1;
      #pragma unroll
      for (int ib = 0; ib < 3; ++ib) {
        #pragma unroll
        for (int ic = 0; ic < (NA == 3 ? 3 : 1); ++ic) {
          int p[3] = {i, j, k}, q[3] = {i, j, k};
          p[ax] += 1;
          q[ax] -= 1;
          p[o1] += ib - 1;
          q[o1] += ib - 1;
          if (NA == 3) {
            p[o2] += ic - 1;
            q[o2] += ic - 1;
          }
          const double wt = NA == 3 ? w[ib] * w[ic] : w[ib];
          acc += wt * (geo_alpha(g, a, p[0], p[1], p[2]) - geo_alpha(g, a, q[0], q[1], q[2]));
        }
      }
      n[ax] = -acc;
    }
    beta = geo_plane_constant(NA, n[0], n[1], n[2], ac);
  }
  N0[id] = n[0];
  N1[id] = n[1];
  if (NA == 3) N2[id] = n[2];
  B[id] = beta;
}

// Liquid passed in the sweep by the face of direction K at face coordinates f: phi_f =
// u_f A_f dt times the fraction of the donor's slab (width |u_f| dt / h) on the liquid side
// of its plane; a full donor passes phi_f, an empty one or one outside the domain nothing,
// one whose normal vanishes its own alpha.  Returns phi_f through *phi.
template <int NA, int K>
__device__ double geo_face_flux(const Geo& g, const Phys& p, const double* a, const double* N0, const double* N1,
                                const double* N2, const double* B, const double* uk, int f0, int f1, int f2,
                                double* phi_out) {
  const double u = uk[fidx(g, K, f0, f1, f2)];
  const double dt = dt_of(p);
  const double phi = u * faceA(g, K, f0) * dt;
  *phi_out = phi;
  const bool pos = phi >= 0.0;
  int d[3] = {f0, f1, f2};
  if (pos) d[K] -= 1;
  if (d[K] < 0 || d[K] >= g.n[K]) return 0.0;
  const long long q = cidx(g, d[0], d[1], d[2]);
  const double ad = iclamp01(a[q]);
  if (ad >= 1.0) return phi;
  if (ad <= 0.0) return 0.0;
  double n[3] = {N0[q], N1[q], NA == 3 ? N2[q] : 0.0};
  if (n[0] == 0.0 && n[1] == 0.0 && n[2] == 0.0) return phi * ad;
  const double c = fmin(fabs(u) * dt / g.h[K], 1.0);
  const double nk = n[K];
  n[K] = c * nk;
  const double bs = pos ? B[q] - nk * (1.0 - c) : B[q];
  return phi * geo_cut_fraction(NA, n[0], n[1], n[2], bs);
}

// sweep K of cell (i, j, k): alpha - (F_hi - F_lo)/V + a_c (dphi_K - dphi / D)/V, a_c = 1
// where alpha* > 1/2; the cell's mean divergence is taken out of each sweep, so the terms
// cancel over the sweeps and the liquid volume is conserved whatever div u is
template <int NA, int K>
__device__ __forceinline__ double geo_sweep_cell(const Geo& g, const Phys& p, const double* a, const double* astar,
                                                 const double* N0, const double* N1, const double* N2, const double* B,
                                                 const double* const U[3], int i, int j, int k, long long id) {
  double phiK_lo, phiK_hi;
  int hi[3] = {i, j, k};
  hi[K] += 1;
  const double Flo = geo_face_flux<NA, K>(g, p, a, N0, N1, N2, B, U[K], i, j, k, &phiK_lo);
  const double Fhi = geo_face_flux<NA, K>(g, p, a, N0, N1, N2, B, U[K], hi[0], hi[1], hi[2], &phiK_hi);
  const double dt = dt_of(p);
  double div = 0.0;
  #pragma unroll
  for (int ax = 0; ax < NA; ++ax) {
    int h2[3] = {i, j, k};
    h2[ax] += 1;
    const double plo = U[ax][fidx(g, ax, i, j, k)] * faceA(g, ax, i) * dt;
    const double phi2 = U[ax][fidx(g, ax, h2[0], h2[1], h2[2])] * faceA(g, ax, h2[0]) * dt;
    div += phi2 - plo;
  }
  const double V = cellV(g, i);
  const double acw = astar[id] > 0.5 ? 1.0 : 0.0;
  return a[id] - (Fhi - Flo) / V + acw * ((phiK_hi - phiK_lo) - div / (double)NA) / V;
}

template <int NA, int K>
__global__ void k_geo_sweep(Geo g, Phys p, const double* a, const double* astar, const double* N0, const double* N1,
                            const double* N2, const double* B, const double* u0, const double* u1, const double* u2,
                            double* out) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  int i, j, k;
  decomp(id, g.n[0], g.n[1], i, j, k);
  const double* U[3] = {u0, u1, u2};
  out[id] = geo_sweep_cell<NA, K>(g, p, a, astar, N0, N1, N2, B, U, i, j, k, id);
}

// the last sweep: clip into [0, 1] with the clipped volume and count summed per block
// (reading R14), mixture properties of alpha^{n+1} (S4)
template <int NA, int K>
__global__ void __launch_bounds__(TPB, 4) k_geo_sweep_last(Geo g, Phys p, const double* a, const double* astar,
                                                           const double* N0, const double* N1, const double* N2,
                                                           const double* B, const double* u0, const double* u1,
                                                           const double* u2, double* alpha, double* partials,
                                                           PropsOut po) {
  double acc[2] = {0.0, 0.0};
  const double* U[3] = {u0, u1, u2};
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < g.N; id += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    decomp(id, g.n[0], g.n[1], i, j, k);
    const double an = geo_sweep_cell<NA, K>(g, p, a, astar, N0, N1, N2, B, U, i, j, k, id);
    const double ac = iclamp01(an);
    if (ac != an) { acc[1] += 1.0; acc[0] += (an - ac) * cellV(g, i); }
    alpha[id] = ac;
    props_out(p, id, ac, po);
  }
  block_sum_store<2>(acc, partials);
}

__global__ void k_clip_finish(const double* partials, int nblk, double* scal, unsigned* flags) {
  double v = block_sum_partials(partials, nblk);
  double c = block_sum_partials(partials + nblk, nblk);
  if (threadIdx.x == 0) {
    scal[SC_CLIP] += v;
    if (c > 0.0) atomicOr(flags, (unsigned)DROPLET_FLAG_ALPHA_CLIPPED);
  }
}

// no advection: clip alpha* into alpha
__global__ void k_alpha_clip_only(Geo g, Phys p, const double* as, double* alpha, double* partials, PropsOut po) {
  double acc[2] = {0.0, 0.0};
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < g.N; id += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    decomp(id, g.n[0], g.n[1], i, j, k);
    double an = as[id], ac = iclamp01(an);
    if (ac != an) { acc[1] += 1.0; acc[0] += (an - ac) * cellV(g, i); }
    alpha[id] = ac;
    props_out(p, id, ac, po);
  }
  block_sum_store<2>(acc, partials);
}

// ============================================================== S5 / S6 scalar transport systems
// coef V (phi - phi^n)/dt + coef [sum F phi_f - phi_P sum F] = sum gamma_f A (phi_N - phi_P)/h + src V
// Box operator: y_P = D_P x_P + sum c (x_P - x_Q); c stored at the high cell of each pair.
// mode 0: energy (coef = rho cp, gamma = k, src = -mdot L), mode 1: species (coef = rho,
// gamma = rho D, rows with alpha >= 1/2 pinned to Y_eq(T^{n+1})).
__device__ __forceinline__ double gam(int mode, const double* kc, const double* rho, const double* D, long long q) {
  return mode == 0 ? kc[q] : rho[q] * D[q];
}
// (FIB, with the fibre: two zero values, the faces between two of its cells, give 0; the sum
// is tested on the integer pipe)
template <bool FIB = false>
__device__ __forceinline__ double harm(double x, double y) {
  const double t = x + y;
  if (FIB && (__double_as_longlong(t) << 1) == 0) return 0.0;
  return 2.0 * x * y * rcp64(t);
}
// half the harmonic mean, x y / (x + y) (the 2 folded into a host constant)
template <bool FIB = false>
__device__ __forceinline__ double harm_half(double x, double y) {
  const double t = x + y;
  if (FIB && (__double_as_longlong(t) << 1) == 0) return 0.0;
  return x * y * rcp64(t);
}

// FIB: with the fibre (zero k and rho D in its cells close the sphere; far upwind values inside
// it replaced by the near ones).  HD (energy rows, c_p,v != c_p,g): the species-diffusion
// enthalpy term of Eq. Teqn, (c_p,v - c_p,g) rho D grad(omega) . grad(T) integrated over the
// cell as half the sum over its interior faces of the species equation's coupling
// harm(rho D) A / h times (omega_N - omega_P)(T_N - T_P), at omega^n = wq and T^n = phi
template <int NA, bool FIB, bool HD = false>
__global__ void k_scalar_assemble(Geo g, Phys p, int mode, const double* phi, const double* rho, const double* cp,
                                  const double* kc, const double* D, const double* mdot, const double* u0,
                                  const double* u1, const double* u2, const double* alpha_new, const double* pinv,
                                  double amb, double* Dg, double* c0, double* c1, double* c2, double* rhs,
                                  const double* wq) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  int i, j, k;
  decomp(id, g.n[0], g.n[1], i, j, k);
  constexpr int na = NA;
  const double* U[3] = {u0, u1, u2};
  double* C[3] = {c0, c1, c2};
  double V = cellV(g, i);
  double coef = mode == 0 ? rho[id] * cp[id] : rho[id];
  double dP = coef * V * idt_of(p);
  const double phiP = phi[id];
  double r = dP * phiP + (mode == 0 ? -mdot[id] * p.Lv : 0.0) * V;
  // the convection sum of phi_f - phi_P over the faces (outward flux sign), i.e.
  // sum F phi_f - phi_P sum F
  double net = 0.0;
  double gP = gam(mode, kc, rho, D, id);
  bool pin = (mode == 1) && ige64(alpha_new[id], 0.5);
  int ci[3] = {i, j, k};
  double hq = 0.0, gdP = 0.0, wP = 0.0;   // HD: the face sum, rho D and omega of the cell
  if (HD) {
    gdP = rho[id] * D[id];
    wP = wq[id];
  }
  #pragma unroll
  for (int a = 0; a < na; ++a) {
    if (HD) {
      if (ci[a] > 0) {
        int Lc[3] = {i, j, k};
        Lc[a] -= 1;
        const long long li = cidx(g, Lc[0], Lc[1], Lc[2]);
        const double cf = NA == 3 ? harm_half<FIB>(rho[li] * D[li], gdP) * g.aih2[a]
                                  : harm<FIB>(rho[li] * D[li], gdP) * faceA(g, a, i) * g.ih[a];
        hq = fma(cf * (wq[li] - wP), phi[li] - phiP, hq);
      }
      if (ci[a] < g.n[a] - 1) {
        int Hc[3] = {i, j, k};
        Hc[a] += 1;
        const long long hi = cidx(g, Hc[0], Hc[1], Hc[2]);
        const double cf = NA == 3 ? harm_half<FIB>(gdP, rho[hi] * D[hi]) * g.aih2[a]
                                  : harm<FIB>(gdP, rho[hi] * D[hi]) * faceA(g, a, Hc[0]) * g.ih[a];
        hq = fma(cf * (wq[hi] - wP), phi[hi] - phiP, hq);
      }
    }
    #pragma unroll
    for (int side = 0; side < 2; ++side) {
      int f[3] = {i, j, k};
      if (side) f[a] += 1;
      double F = U[a][fidx(g, a, f[0], f[1], f[2])] * faceA(g, a, f[0]);
      double val;
      if (f[a] == 0 || f[a] == g.n[a]) {
        int kind = (side ? g.bc[a][1] : g.bc[a][0]);
        bool inflow = side == 0 ? (F > 0.0) : (F < 0.0);
        val = ((kind == BC_OPEN || kind == BC_FORCED) && inflow) ? amb : phiP;
      } else {
        int L[3] = {f[0], f[1], f[2]};
        L[a] -= 1;
        int LL[3] = {L[0], L[1], L[2]}, RR[3] = {f[0], f[1], f[2]};
        LL[a] -= 1;
        RR[a] += 1;
        double vL = phi[cidx(g, L[0], L[1], L[2])], vR = phi[cidx(g, f[0], f[1], f[2])];
        // the upwind side's operands chosen by the sign bit of F (integer selects, one
        // limited value; a zero F multiplies it either way)
        const bool pos = __double_as_longlong(F) >= 0;
        double far = pos ? cellg(g, phi, LL[0], LL[1], LL[2], R_TO, amb, u0, u1, u2)
                         : cellg(g, phi, RR[0], RR[1], RR[2], R_TO, amb, u0, u1, u2);
        // a far upwind cell inside the fibre: the near one's value (zero gradient)
        if (FIB && (pos ? solid_nb(g, LL[0], LL[1], LL[2]) : solid_nb(g, RR[0], RR[1], RR[2]))) far = pos ? vL : vR;
        val = lim_up(far, pos ? vL : vR, pos ? vR : vL);
      }
      net = fma(side ? F : -F, val - phiP, net);
    }
    // coupling across the low face, stored at this cell
    double cl = 0.0;
    if (ci[a] > 0) {
      int Lc[3] = {i, j, k};
      Lc[a] -= 1;
      long long li = cidx(g, Lc[0], Lc[1], Lc[2]);
      cl = NA == 3 ? harm_half<FIB>(gam(mode, kc, rho, D, li), gP) * g.aih2[a]
                   : harm<FIB>(gam(mode, kc, rho, D, li), gP) * faceA(g, a, i) * g.ih[a];
      if (mode == 1) {
        bool lp = ige64(alpha_new[li], 0.5);
        if (!pin && lp) { r += cl * pinv[li]; dP += cl; }
        if (pin || lp) cl = 0.0;
      }
    }
    C[a][id] = cl;
    // coupling across the high face (owned by the neighbour): only the pinned-neighbour transfer here
    if (mode == 1 && ci[a] < g.n[a] - 1 && !pin) {
      int Hc[3] = {i, j, k};
      Hc[a] += 1;
      long long hi = cidx(g, Hc[0], Hc[1], Hc[2]);
      if (ige64(alpha_new[hi], 0.5)) {
        double ch = NA == 3 ? harm_half<FIB>(gP, gam(mode, kc, rho, D, hi)) * g.aih2[a]
                            : harm<FIB>(gP, gam(mode, kc, rho, D, hi)) * faceA(g, a, Hc[0]) * g.ih[a];
        r += ch * pinv[hi];
        dP += ch;
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
        double cb = gP * faceA(g, a, f[0]) * (2.0 * g.ih[a]);
        dP += cb;
        r += cb * amb;
      }
    }
  }
  r -= coef * net;
  if (HD) r = fma(0.5 * (p.cp_v - p.cp_g), hq, r);
  if (pin) {
    // pinned row, scaled like the other rows: (coef V/dt) x = (coef V/dt) Y_eq
    double dd = coef * V * idt_of(p);
    r = dd * pinv[id];
    dP = dd;
  }
  Dg[id] = dP;
  rhs[id] = r;
}

// saturation value for the rows pinned in the species solve (alpha >= 1/2); 0 elsewhere (unused)
__global__ void k_yeq(Geo g, Phys p, const double* T, const double* alpha, const double* omega, double* yq,
                      unsigned* flags) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  if (alpha[id] < 0.5) { yq[id] = 0.0; return; }
  unsigned b = 0;
  yq[id] = Y_eq(p, T[id], &b, omega[id]);
  if (b) atomicOr(flags, (unsigned)DROPLET_FLAG_BOILING);
}

__global__ void k_species_noflow(Geo g, const double* alpha_new, const double* yq, double* omega) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  if (ige64(alpha_new[id], 0.5)) omega[id] = yq[id];
}

__global__ void k_rhoG(Geo g, Phys p, const double* T, const double* w, double* rhoG) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  rhoG[id] = rho_gas(p, T[id], w[id]);
}

// ============================================================== S7 momentum predictor
// For each interior face of direction c (box index b, face index f = b + e_c),
// V_f-weighted: rho_f V_f/dt u* - [implicit viscous] = rho_f V_f u^n/dt + adv + visc^T + forces.
// muLR = mu_L + mu_R of the face's two cells, shared by its edges (the sum in the same order)
__device__ __forceinline__ double mu_edge(const Geo& g, const double* mu, double muLR, const int L[3], const int R[3],
                                          int a, int sh) {
  int La[3] = {L[0], L[1], L[2]}, Ra[3] = {R[0], R[1], R[2]};
  La[a] += sh;
  Ra[a] += sh;
  double s = muLR + cellc(g, mu, La[0], La[1], La[2]) + cellc(g, mu, Ra[0], Ra[1], Ra[2]);
  return 0.25 * s;
}

// FIB: with the fibre, whose faces are pinned at u* = 0 (no slip, no penetration) and whose
// neighbouring faces take their coupling to them into the diagonal (the known value 0)
template <int C, int NA, bool FIB>
__global__ void k_mom_assemble(Geo g, Phys p, const double* u0, const double* u1, const double* u2,
                               const double* rho, const double* mu, const double* pr, const double* alpha,
                               const double* xi, double* Dg, double* c0, double* c1, double* c2, double* rhs) {
  constexpr int c = C;
  constexpr bool cart = NA == 3;   // 3D grids are Cartesian, 2D ones axisymmetric
  // box dims: n with n_c - 1 along c
  int m[3] = {g.n[0], g.n[1], g.n[2]};
  m[c] -= 1;
  long long nb = (long long)m[0] * m[1] * m[2];
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= nb) return;
  int b[3];
  decomp(id, m[0], m[1], b[0], b[1], b[2]);
  int f[3] = {b[0], b[1], b[2]};
  f[c] += 1;                                   // face index
  int L[3] = {f[0], f[1], f[2]}, R[3] = {f[0], f[1], f[2]};
  L[c] -= 1;
  const double* U[3] = {u0, u1, u2};
  const double* uc = U[c];
  double* Cc[3] = {c0, c1, c2};
  constexpr int na = NA;
  long long li = cidx(g, L[0], L[1], L[2]), ri = cidx(g, R[0], R[1], R[2]);
  double rhoL = rho[li], rhoR = rho[ri], muL = mu[li], muR = mu[ri];
  // rho_f V_f with rho_f the mean of the two cells, and the face area
  double r_f = 0.0, V_f, rV, A_f;
  if (cart) {
    V_f = g.vol3;
    rV = (rhoL + rhoR) * g.hvol3;
    A_f = g.area3[c];
  } else {
    r_f = (c == 0) ? f[0] * g.h[0] : (f[0] + 0.5) * g.h[0];
    V_f = r_f * g.h[0] * g.h[1];
    rV = 0.5 * (rhoL + rhoR) * V_f;
    A_f = V_f * g.ih[c];
  }
  double u_f = uc[fidx(g, c, f[0], f[1], f[2])];
  const double muLR = muL + muR;
  double d = rV * idt_of(p);
  if (FIB && sphere_face(g, c, f[0], f[1], f[2])) {   // a face of the sphere: a decoupled row, u* = 0
    Dg[id] = d;
    rhs[id] = 0.0;
    #pragma unroll
    for (int a = 0; a < NA; ++a) Cc[a][id] = 0.0;
    return;
  }
  double r = d * u_f;
  // advection accumulated without its common factor -rho_f V_f
  double s_adv = 0.0, t_vT = 0.0, d_visc = 0.0;
  #pragma unroll
  for (int a = 0; a < na; ++a) {
    // ---- advection (advective form, minmod limited linear upwind)
    // ubs: the advecting velocity, for a != c four times it (the mean of the four
    // surrounding faces of direction a; its quarter is folded into the factor qih)
    double ubs, uaL_lo = 0.0, uaL_hi = 0.0, uaR_lo = 0.0, uaR_hi = 0.0;
    if (a == c) ubs = u_f;
    else {
      const double* ua = U[a];
      int La[3] = {L[0], L[1], L[2]}, Ra[3] = {R[0], R[1], R[2]};
      La[a] += 1;
      Ra[a] += 1;
      uaL_lo = ua[fidx(g, a, L[0], L[1], L[2])];
      uaL_hi = ua[fidx(g, a, La[0], La[1], La[2])];
      uaR_lo = ua[fidx(g, a, R[0], R[1], R[2])];
      uaR_hi = ua[fidx(g, a, Ra[0], Ra[1], Ra[2])];
      ubs = ((uaL_lo + uaL_hi) + uaR_lo) + uaR_hi;
    }
    int q[3];
    double us[5];
    #pragma unroll
    for (int s = -2; s <= 2; ++s) {
      q[0] = f[0]; q[1] = f[1]; q[2] = f[2];
      q[a] += s;
      us[s + 2] = ufg(g, uc, c, q[0], q[1], q[2]);
    }
    // u(+1/2) - u(-1/2) of the limited upwind values, without a branch: with the differences
    // d_k = us[k] - us[k-1] and M = minmod(d21, d32), it is d21 + (M - minmod(d10, d21)) / 2
    // for ubar >= 0 and d32 + (M - minmod(d32, d43)) / 2 otherwise (the sign taken from the
    // sign bit on the integer pipe: a zero ubar multiplies the difference either way)
    const double d10 = us[1] - us[0], d21 = us[2] - us[1], d32 = us[3] - us[2], d43 = us[4] - us[3];
    const bool pos = __double_as_longlong(ubs) >= 0;
    const double M2 = minmod(d21, d32);
    const double X = pos ? minmod(d10, d21) : minmod(d32, d43);
    const double dd = fma(0.5, M2 - X, pos ? d21 : d32);
    s_adv = fma(ubs * dd, a == c ? g.ih[a] : g.qih[a], s_adv);
    // ---- viscous
    if (a == c) {
      double kR, kL;
      if (cart) {
        kR = muR * g.aih[c];
        kL = muL * g.aih[c];
      } else {
        double ApL, ApR;
        if (c == 0) { ApL = areaN(g, 0, (L[0] + 0.5) * g.h[0]); ApR = areaN(g, 0, (R[0] + 0.5) * g.h[0]); }
        else { ApL = ApR = areaN(g, 1, r_f); }
        kR = muR * (ApR * g.ih[c]);
        kL = muL * (ApL * g.ih[c]);
      }
      t_vT = t_vT + (kR * d32 - kL * d21);
      // coupling with the lower neighbour face (stored at this box cell)
      Cc[c][id] = (b[c] > 0) ? kL : 0.0;
      if (b[c] == 0 && g.bc[c][0] != BC_OPEN) {
        int fb[3] = {f[0], f[1], f[2]};
        fb[c] = 0;
        d_visc += kL;
        r += kL * uc[fidx(g, c, fb[0], fb[1], fb[2])];
      }
      if (b[c] == m[c] - 1 && g.bc[c][1] != BC_OPEN) {
        int fb[3] = {f[0], f[1], f[2]};
        fb[c] = g.n[c];
        d_visc += kR;
        r += kR * uc[fidx(g, c, fb[0], fb[1], fb[2])];
      }
      if (FIB) {   // neighbour faces along c on the sphere
        if (b[c] > 0 && sphere_face(g, c, f[0] - (c == 0), f[1] - (c == 1), f[2] - (c == 2))) {
          Cc[c][id] = 0.0;
          d_visc += kL;
        }
        if (b[c] < m[c] - 1 && sphere_face(g, c, f[0] + (c == 0), f[1] + (c == 1), f[2] + (c == 2))) d_visc += kR;
      }
    } else {
      double kp, km;
      if (cart) {
        // edge viscosities as sums of their four cells, the quarter in the constants
        int La[3] = {L[0], L[1], L[2]}, Ra[3] = {R[0], R[1], R[2]};
        La[a] += 1;
        Ra[a] += 1;
        const double sp = muLR + cellc(g, mu, La[0], La[1], La[2]) + cellc(g, mu, Ra[0], Ra[1], Ra[2]);
        La[a] -= 2;
        Ra[a] -= 2;
        const double sm = muLR + cellc(g, mu, La[0], La[1], La[2]) + cellc(g, mu, Ra[0], Ra[1], Ra[2]);
        kp = sp * g.qaih[a];
        km = sm * g.qaih[a];
        t_vT = t_vT + (sp * (uaR_hi - uaL_hi) - sm * (uaR_lo - uaL_lo)) * g.qvt[c][a];
      } else {
        double App, Apm;
        if (a == 0) { App = areaN(g, 0, (f[0] + 1) * g.h[0]); Apm = areaN(g, 0, f[0] * g.h[0]); }
        else { App = Apm = areaN(g, 1, r_f); }
        double mup = mu_edge(g, mu, muLR, L, R, a, 1), mum = mu_edge(g, mu, muLR, L, R, a, -1);
        kp = mup * (App * g.ih[a]);
        km = mum * (Apm * g.ih[a]);
        t_vT = t_vT + (mup * App * (uaR_hi - uaL_hi) - mum * Apm * (uaR_lo - uaL_lo)) * g.ih[c];
      }
      Cc[a][id] = (b[a] > 0) ? km : 0.0;
      if (b[a] == 0 && (g.bc[a][0] == BC_WALL || g.bc[a][0] == BC_FORCED)) d_visc += 2.0 * km;
      if (b[a] == m[a] - 1 && (g.bc[a][1] == BC_WALL || g.bc[a][1] == BC_FORCED)) d_visc += 2.0 * kp;
      if (FIB) {   // neighbour faces along a on the sphere
        if (b[a] > 0 && sphere_face(g, c, f[0] - (a == 0), f[1] - (a == 1), f[2] - (a == 2))) {
          Cc[a][id] = 0.0;
          d_visc += km;
        }
        if (b[a] < m[a] - 1 && sphere_face(g, c, f[0] + (a == 0), f[1] + (a == 1), f[2] + (a == 2))) d_visc += kp;
      }
    }
  }
  if (!cart && c == 0 && r_f > 0.0) d_visc = d_visc + 2.0 * (0.5 * muLR) * V_f / (r_f * r_f);
  // pressure, buoyancy and centripetal force in the balanced face form; g . x from the
  // host-formed constants (axes without gravity skipped: a uniform branch)
  double gx = g.gxc[c];
  #pragma unroll
  for (int a = 0; a < na; ++a)
    if (g.gmask >> a & 1) gx = fma(g.gh[a], (double)f[a], gx);
  double xiL = xi[li], xiR = xi[ri];
  double raL = rhoL * alpha[li], raR = rhoR * alpha[ri];
  double t_force = A_f * ((0.5 * (raL + raR) * (xiR - xiL) - gx * (rhoR - rhoL)) - (pr[ri] - pr[li]));
  d = d + d_visc;
  r = r - rV * s_adv + t_vT + t_force;
  Dg[id] = d;
  rhs[id] = r;
}

// u* of direction c from the box solution; boundary faces by their rule.
template <int C>
__global__ void k_mom_scatter(Geo g, Phys p, const double* x, double* us) {
  constexpr int c = C;
  long long nf = nfaces(g, c);
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= nf) return;
  int m0 = g.n[0] + (c == 0), m1 = g.n[1] + (c == 1);
  int f[3];
  decomp(id, m0, m1, f[0], f[1], f[2]);
  int mb[3] = {g.n[0], g.n[1], g.n[2]};
  mb[c] -= 1;
  auto box = [&](int fc) {
    int b[3] = {f[0], f[1], f[2]};
    b[c] = fc - 1;
    return x[(long long)b[0] + (long long)mb[0] * ((long long)b[1] + (long long)mb[1] * b[2])];
  };
  if (f[c] > 0 && f[c] < g.n[c]) {
    // (a face of the fibre's sphere: exactly 0, the value its decoupled row solves for)
    us[id] = sphere_face(g, c, f[0], f[1], f[2]) ? 0.0 : box(f[c]);
    return;
  }
  int side = f[c] == 0 ? 0 : 1;
  int kind = (side ? g.bc[c][1] : g.bc[c][0]);
  if (kind == BC_OPEN) us[id] = box(side ? g.n[c] - 1 : 1);
  // axis / wall: stays 0; forced inlet: keeps u_in (both already stored)
}

// Initial guess of a Helmholtz solve: the linear extrapolation in time x^n + (x^n -
// x^{n-1}) where the previous step's field is held (scal[SC_HIST] = 1), else x^n; the
// history then takes x^n.  Only the starting point of the iteration changes: the
// solution is the system's, to the solver's tolerance, either way.
__global__ void k_extrap(long long n, double* x, double* xh, const double* scal) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= n) return;
  const double v = x[id];
  if (scal[SC_HIST] != 0.0) x[id] = 2.0 * v - xh[id];
  xh[id] = v;
}

// initial guess of the momentum solve of direction c on the interior faces: u^n,
// extrapolated in time as in k_extrap (history uh on the faces)
template <int C>
__global__ void k_faces_to_box(Geo g, const double* u, double* x, double* uh, const double* scal) {
  constexpr int c = C;
  int m[3] = {g.n[0], g.n[1], g.n[2]};
  m[c] -= 1;
  long long nb = (long long)m[0] * m[1] * m[2];
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= nb) return;
  int b[3];
  decomp(id, m[0], m[1], b[0], b[1], b[2]);
  b[c] += 1;
  const long long f = fidx(g, c, b[0], b[1], b[2]);
  const double v = u[f];
  x[id] = scal[SC_HIST] != 0.0 ? 2.0 * v - uh[f] : v;
  uh[f] = v;
}

// ============================================================== S8 - S10 projection
// S = mdot (1/rho_G - 1/rho_L) - (1 - alpha)/rho_G [(rho_G^{n+1} - rho_G^n)/dt + vbar . grad rho_G^{n+1}]
//     - E,  E = alpha/rho_L [(rho_L^{n+1} - rho_L^n)/dt + vbar . grad rho_L^{n+1}]
// sum beta_f (dp_P - dp_N) + sum_open beta_b dp_P = (S V - sum u* A)/dt
// The liquid's expansion term E (a temperature-dependent liquid density, rho_L^n = rho_L(T^n)
// from T0, rho_L^{n+1} from T1) is formed when `expand` is given, and stored there: the next
// step's alpha source subtracts it, so that in the liquid it cancels the divergence it puts
// into the advecting velocity.
template <int NA>
__global__ void k_poisson_assemble(Geo g, Phys p, const double* mdot, const double* alpha, const double* rgo,
                                   const double* rgn, const double* u0, const double* u1, const double* u2,
                                   const double* us0, const double* us1, const double* us2, const double* rho,
                                   const double* T1, const double* T0, double* expand,
                                   double* S, double* Dg, double* c0, double* c1, double* c2, double* rhs,
                                   double* dp0) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= g.N) return;
  dp0[id] = 0.0;   // the solve's zero initial guess
  int i, j, k;
  decomp(id, g.n[0], g.n[1], i, j, k);
  constexpr int na = NA;
  const double* U[3] = {u0, u1, u2};
  const double* US[3] = {us0, us1, us2};
  double* C[3] = {c0, c1, c2};
  int ci[3] = {i, j, k};
  double adv = 0.0, advl = 0.0;
  #pragma unroll
  for (int a = 0; a < na; ++a) {
    int hi[3] = {i, j, k};
    hi[a] += 1;
    double vc = 0.5 * (U[a][fidx(g, a, i, j, k)] + U[a][fidx(g, a, hi[0], hi[1], hi[2])]);
    int qp[3] = {i, j, k}, qm[3] = {i, j, k};
    qp[a] += 1;
    qm[a] -= 1;
    double rgp = cellg(g, rgn, qp[0], qp[1], qp[2], R_ZG, 0, 0, 0, 0), rgm = cellg(g, rgn, qm[0], qm[1], qm[2], R_ZG, 0, 0, 0, 0);
    if (g.fib) {   // zero gradient across the fibre's sphere
      if (solid_nb(g, qp[0], qp[1], qp[2])) rgp = rgn[id];
      if (solid_nb(g, qm[0], qm[1], qm[2])) rgm = rgn[id];
    }
    double gr = (rgp - rgm) * (0.5 * g.ih[a]);
    adv = adv + vc * gr;
    if (expand) {   // rho_L(T^{n+1}) with zero-gradient ghosts: the liquid density of the ghost temperature
      double gl = (rho_liq(p, cellg(g, T1, qp[0], qp[1], qp[2], R_ZG, 0, 0, 0, 0)) -
                   rho_liq(p, cellg(g, T1, qm[0], qm[1], qm[2], R_ZG, 0, 0, 0, 0))) * (0.5 * g.ih[a]);
      advl = advl + vc * gl;
    }
  }
  double rn = rgn[id], irn = rcp64(rn);
  double s;
  if (expand) {
    const double rl1 = rho_liq(p, T1[id]), rl0 = rho_liq(p, T0[id]);
    const double e = alpha[id] / rl1 * ((rl1 - rl0) * idt_of(p) + advl);
    expand[id] = e;
    s = mdot[id] * (irn - 1.0 / rl1) - (1.0 - alpha[id]) * irn * ((rn - rgo[id]) * idt_of(p) + adv) - e;
  } else {
    s = mdot[id] * (irn - p.irho_l) - (1.0 - alpha[id]) * irn * ((rn - rgo[id]) * idt_of(p) + adv);
  }
  const bool sol = solid_cell(g, id);
  if (sol) s = 0.0;   // the fibre holds no fluid: no continuity source
  S[id] = s;
  double dg = 0.0, div = 0.0;
  double rP = rho[id];
  #pragma unroll
  for (int a = 0; a < na; ++a) {
    int hi[3] = {i, j, k};
    hi[a] += 1;
    div += US[a][fidx(g, a, hi[0], hi[1], hi[2])] * faceA(g, a, hi[0]) - US[a][fidx(g, a, i, j, k)] * faceA(g, a, i);
    double cl = 0.0;
    if (ci[a] > 0) {
      int Lc[3] = {i, j, k};
      Lc[a] -= 1;
      // A / h over the mean density of the two cells (3D: 2 A / h from the host)
      const long long li = cidx(g, Lc[0], Lc[1], Lc[2]);
      const double ir = rcp64(rho[li] + rP);
      cl = NA == 3 ? g.aih2[a] * ir : faceA(g, a, i) * g.ih[a] * (2.0 * ir);
      if (g.fib && (sol || g.solid[li])) cl = 0.0;   // a face of the sphere: zero normal gradient
    }
    C[a][id] = cl;
    if (ci[a] == 0 && g.bc[a][0] == BC_OPEN) dg += faceA(g, a, i) * (2.0 * g.ih[a]) / rP;
    if (ci[a] == g.n[a] - 1 && g.bc[a][1] == BC_OPEN) dg += faceA(g, a, hi[0]) * (2.0 * g.ih[a]) / rP;
  }
  // a cell of the fibre: a decoupled row (its increment is 0), of the size of the surrounding
  // liquid's Laplacian diagonal, 2 d V / (h_min^2 rho_L) (a larger one anchors the coarse cells
  // of the multigrid that contain it and slows the pressure solve)
  if (sol) dg = 2.0 * na * cellV(g, i) / (g.hmin * g.hmin * p.rho_l);
  Dg[id] = dg;
  rhs[id] = (s * cellV(g, i) - div) * idt_of(p);
}

// u = u* - dt beta_f (dp_R - dp_L)/A_f with dp = 0 beyond open faces (half-cell distance);
// beta_f / A_f = 1 / (h rho_f)
template <int C>
__device__ __forceinline__ void correct_face(const Geo& g, const Phys& p, const double* us, const double* dp,
                                             const double* rho, double* u, long long id) {
  constexpr int c = C;
  int m0 = g.n[0] + (c == 0), m1 = g.n[1] + (c == 1);
  int f[3];
  decomp(id, m0, m1, f[0], f[1], f[2]);
  double A = faceA(g, c, f[0]);
  double corr = 0.0;
  if (__double_as_longlong(A) > 0) {   // A > 0 (areas are never negative), on the integer pipe
    int L[3] = {f[0], f[1], f[2]};
    L[c] -= 1;
    if (f[c] > 0 && f[c] < g.n[c]) {
      long long li = cidx(g, L[0], L[1], L[2]), ri = cidx(g, f[0], f[1], f[2]);
      corr = (dt_of(p) * g.ih[c]) * (2.0 * rcp64(rho[li] + rho[ri])) * (dp[ri] - dp[li]);
      if (g.fib && (g.solid[li] || g.solid[ri])) corr = 0.0;   // the sphere's faces keep u* = 0
    } else {
      int side = f[c] == 0 ? 0 : 1;
      if ((side ? g.bc[c][1] : g.bc[c][0]) == BC_OPEN) {
        long long pi = side ? cidx(g, L[0], L[1], L[2]) : cidx(g, f[0], f[1], f[2]);
        const double bA = (2.0 * g.ih[c]) * rcp64(rho[pi]);
        corr = side ? dt_of(p) * bA * (0.0 - dp[pi]) : dt_of(p) * bA * (dp[pi] - 0.0);
      }
    }
  }
  u[id] = us[id] - corr;
}

template <int C>
__global__ void k_correct(Geo g, Phys p, const double* us, const double* dp, const double* rho, double* u) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= nfaces(g, C)) return;
  correct_face<C>(g, p, us, dp, rho, u, id);
}

// every direction's correction and p_rgh += dp, one launch: blocks [0, b0) take the faces
// of direction 0, then direction 1 (and 2), then the cells
struct CorrectArgs {
  const double* us[3];
  double* u[3];
  const double *dp, *rho;
  double* pr;
  int b[4];   // first block of each segment (directions, then cells)
};
__global__ void k_correct_all(Geo g, Phys p, CorrectArgs a) {
  const int bx = blockIdx.x;
  if (bx < a.b[1]) {
    long long id = (long long)(bx - a.b[0]) * blockDim.x + threadIdx.x;
    if (id < nfaces(g, 0)) correct_face<0>(g, p, a.us[0], a.dp, a.rho, a.u[0], id);
  } else if (bx < a.b[2]) {
    long long id = (long long)(bx - a.b[1]) * blockDim.x + threadIdx.x;
    if (id < nfaces(g, 1)) correct_face<1>(g, p, a.us[1], a.dp, a.rho, a.u[1], id);
  } else if (bx < a.b[3]) {
    long long id = (long long)(bx - a.b[2]) * blockDim.x + threadIdx.x;
    if (id < nfaces(g, 2)) correct_face<2>(g, p, a.us[2], a.dp, a.rho, a.u[2], id);
  } else {
    long long id = (long long)(bx - a.b[3]) * blockDim.x + threadIdx.x;
    if (id < g.N) a.pr[id] += a.dp[id];
  }
}

__global__ void k_add(long long n, double* y, const double* x) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id < n) y[id] += x[id];
}

// ============================================================== S11 diagnostics
// sums: alpha V, mdot V, T |grad alpha| V, |grad alpha| V, (1-alpha) rhoG omega V, open-boundary vapour outflow
// maxima: |u|, alpha, -alpha
// Every value read is also tested for NaN / infinity (all exponent bits set, on the
// integer pipe); one is enough to set DROPLET_FLAG_NONFINITE (the max reductions drop NaN).
__device__ __forceinline__ unsigned nonfinite_bits(double x) {
  return (unsigned)((__double_as_longlong(x) & 0x7FF0000000000000LL) == 0x7FF0000000000000LL);
}
template <int NA>
__global__ void __launch_bounds__(TPB, 4) k_diag(Geo g, Phys p, const double* alpha, const double* T, const double* mdot, const double* omega,
                       const double* rhoG, const double* u0, const double* u1, const double* u2, double* psum,
                       double* pmax, unsigned* flags) {
  double s[7] = {0, 0, 0, 0, 0, 0, 0};
  double mx[3] = {0.0, -1e300, -1e300};
  unsigned bad = 0u;
  constexpr int na = NA;
  const double* U[3] = {u0, u1, u2};
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < g.N; id += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    decomp(id, g.n[0], g.n[1], i, j, k);
    double V = cellV(g, i);
    double a = alpha[id];
    bad |= nonfinite_bits(a) | nonfinite_bits(T[id]) | nonfinite_bits(omega[id]) | nonfinite_bits(rhoG[id]) |
           nonfinite_bits(mdot[id]);
    double gr[3];
    s[0] += a * V;
    const double md = mdot[id];
    if (md != 0.0) s[1] += md * V;
    if (!grad_alpha_flat(g, alpha, i, j, k, gr) && !solid_cell(g, id)) {   // (a flat cell adds zeros; the fibre none)
      double gm = sqrt(gr[0] * gr[0] + gr[1] * gr[1] + (g.act3 ? gr[2] * gr[2] : 0.0));
      s[2] += T[id] * gm * V;
      s[3] += gm * V;
    }
    s[4] += (1.0 - a) * rhoG[id] * omega[id] * V;
    if (p.drl != 0.0) s[6] += rho_liq(p, T[id]) * a * V;   // the liquid mass (constant density: rho_l V_l)
    mx[1] = imax64(mx[1], a);
    mx[2] = imax64(mx[2], -a);
    int ci[3] = {i, j, k};
    #pragma unroll
    for (int q = 0; q < na; ++q) {
      const double uq = U[q][fidx(g, q, i, j, k)];
      bad |= nonfinite_bits(uq);
      mx[0] = imax64(mx[0], fabs(uq));
      if (ci[q] == g.n[q] - 1) {
        int hi[3] = {i, j, k};
        hi[q] += 1;
        const double uh = U[q][fidx(g, q, hi[0], hi[1], hi[2])];
        bad |= nonfinite_bits(uh);
        mx[0] = imax64(mx[0], fabs(uh));
      }
      #pragma unroll
      for (int side = 0; side < 2; ++side) {
        bool atb = side ? (ci[q] == g.n[q] - 1) : (ci[q] == 0);
        int kind = (side ? g.bc[q][1] : g.bc[q][0]);
        if (!atb || !(kind == BC_OPEN || kind == BC_FORCED)) continue;
        int f[3] = {i, j, k};
        if (side) f[q] += 1;
        double un = U[q][fidx(g, q, f[0], f[1], f[2])];
        double vout = side ? un : -un;
        if (vout > 0.0) s[5] += rhoG[id] * omega[id] * vout * faceA(g, q, f[0]);
      }
    }
  }
  if (__syncthreads_or((int)bad) && threadIdx.x == 0) atomicOr(flags, (unsigned)DROPLET_FLAG_NONFINITE);
  block_sum_store<7>(s, psum);
  __syncthreads();
  block_max_store<3>(mx, pmax);
}

// mode (DIAG_*): DIAG_STEP_END after a step, whose solves have filled the history fields
// and whose dt advances the clock; then, and for an initial state, a Courant-adaptive run
// (co_hmin = threshold Courant number x h_min > 0) takes its next dt from the face
// velocities just reduced: min(dt_max, co_hmin / max|u|, 1.2 dt) (the growth limit not for
// the first step).
__global__ void k_diag_finish(const double* psum, const double* pmax, int nblk, double* scal, int mode,
                              double co_hmin, double dt_max) {
  double v[7], m[3];
  block_reduce_partials<7, false>(psum, nblk, v);
  block_reduce_partials<3, true>(pmax, nblk, m);
  if (threadIdx.x == 0) {
    scal[SC_SUM_ALPHA_V] = v[0];
    scal[SC_SUM_MDOT_V] = v[1];
    scal[SC_SUM_TG] = v[2];
    scal[SC_SUM_G] = v[3];
    scal[SC_SUM_VAP] = v[4];
    scal[SC_SUM_MLIQ] = v[6];
    scal[SC_VAPOUT] += v[5] * scal[SC_DT];
    scal[SC_MAXU] = m[0];
    scal[SC_AMAX] = m[1];
    scal[SC_AMIN] = -m[2];
    scal[SC_HIST] = mode == DIAG_STEP_END ? 1.0 : 0.0;
    const double dt = scal[SC_DT];
    if (mode == DIAG_STEP_END) scal[SC_TIME] += dt;
    if (co_hmin > 0.0 && mode != DIAG_SET) {
      double d = dt_max;
      if (m[0] > 0.0) d = fmin(d, co_hmin / m[0]);
      if (mode == DIAG_STEP_END) d = fmin(d, 1.2 * dt);
      scal[SC_DT] = d;
      scal[SC_IDT] = 1.0 / d;
    }
  }
}

// ============================================================== launch wrappers
void L_evap_raw(cudaStream_t st, int grid, Geo g, Phys p, const double* alpha, const double* omega, const double* rhoG, const double* T, const double* u0, const double* u1, const double* u2, double* mraw, int* adj, double* partials, unsigned* flags) {
  ++g_launches;
  if (nact(g) == 3) k_evap_raw<3><<<grid, TPB, 0, st>>>(g, p, alpha, omega, rhoG, T, u0, u1, u2, mraw, adj, partials, flags);
  else k_evap_raw<2><<<grid, TPB, 0, st>>>(g, p, alpha, omega, rhoG, T, u0, u1, u2, mraw, adj, partials, flags);
}

void L_adv_faces(cudaStream_t st, int grid, Geo g, Phys p, int a, const double* as, const double* ua, double* FL, double* AF) {
  ++g_launches;
  if (nact(g) == 3) {
    if (a == 0) k_adv_faces<0, 3><<<grid, TPB, 0, st>>>(g, p, as, ua, FL, AF);
    else if (a == 1) k_adv_faces<1, 3><<<grid, TPB, 0, st>>>(g, p, as, ua, FL, AF);
    else k_adv_faces<2, 3><<<grid, TPB, 0, st>>>(g, p, as, ua, FL, AF);
  } else {
    if (a == 0) k_adv_faces<0, 2><<<grid, TPB, 0, st>>>(g, p, as, ua, FL, AF);
    else k_adv_faces<1, 2><<<grid, TPB, 0, st>>>(g, p, as, ua, FL, AF);
  }
}

void L_adv_limit(cudaStream_t st, int grid, Geo g, const double* as, const double* aL, const double* A0, const double* A1, const double* A2, double* Rp, double* Rm) {
  ++g_launches;
  if (nact(g) == 3) k_adv_limit<3><<<grid, TPB, 0, st>>>(g, as, aL, A0, A1, A2, Rp, Rm);
  else k_adv_limit<2><<<grid, TPB, 0, st>>>(g, as, aL, A0, A1, A2, Rp, Rm);
}

void L_adv_update(cudaStream_t st, int grid, Geo g, Phys p, const double* aL, const double* A0, const double* A1, const double* A2, const double* Rp, const double* Rm, double* alpha, double* partials, unsigned* flags, PropsOut po) {
  ++g_launches;
  if (nact(g) == 3) k_adv_update<3><<<grid, TPB, 0, st>>>(g, p, aL, A0, A1, A2, Rp, Rm, alpha, partials, flags, po);
  else k_adv_update<2><<<grid, TPB, 0, st>>>(g, p, aL, A0, A1, A2, Rp, Rm, alpha, partials, flags, po);
}

// geometric advection (S3 with adv_scheme 1): one plane reconstruction and one sweep per
// axis; ping-pong through w[0], w[1] (alpha after sweeps 1 and 2), the last sweep writing
// alpha^{n+1}, its clip partials and the mixture properties
void L_geo_advect(cudaStream_t st, int grid, Geo g, Phys p, const double* astar, double* const w[2],
                  double* const N[3], double* B, double* const u[3], double* alpha, double* partials, PropsOut po) {
  const int na = nact(g), gc = lin_grid(g.N);
  const double* in = astar;
  double* u2 = u[2] ? u[2] : u[0];
  double* n2 = N[2] ? N[2] : N[0];
  for (int s = 0; s < na; ++s) {
    ++g_launches;
    if (na == 3) k_geo_plane<3><<<gc, TPB, 0, st>>>(g, in, N[0], N[1], n2, B);
    else k_geo_plane<2><<<gc, TPB, 0, st>>>(g, in, N[0], N[1], n2, B);
    ++g_launches;
    if (s < na - 1) {
      if (na == 3 && s == 0) k_geo_sweep<3, 0><<<gc, TPB, 0, st>>>(g, p, in, astar, N[0], N[1], n2, B, u[0], u[1], u2, w[s]);
      else if (na == 3) k_geo_sweep<3, 1><<<gc, TPB, 0, st>>>(g, p, in, astar, N[0], N[1], n2, B, u[0], u[1], u2, w[s]);
      else k_geo_sweep<2, 0><<<gc, TPB, 0, st>>>(g, p, in, astar, N[0], N[1], n2, B, u[0], u[1], u2, w[s]);
      in = w[s];
    } else if (na == 3) {
      k_geo_sweep_last<3, 2><<<grid, TPB, 0, st>>>(g, p, in, astar, N[0], N[1], n2, B, u[0], u[1], u2, alpha, partials, po);
    } else {
      k_geo_sweep_last<2, 1><<<grid, TPB, 0, st>>>(g, p, in, astar, N[0], N[1], n2, B, u[0], u[1], u2, alpha, partials, po);
    }
  }
}

void L_scalar_assemble(cudaStream_t st, int grid, Geo g, Phys p, int mode, const double* phi, const double* rho, const double* cp, const double* kc, const double* D, const double* mdot, const double* u0, const double* u1, const double* u2, const double* alpha_new, const double* pinv, double amb, double* Dg, double* c0, double* c1, double* c2, double* rhs, const Shadow32*, const double* wq) {
  ++g_launches;
  // the enthalpy term of the energy rows (wq: omega^n) when the heat capacities differ
  const bool hd = mode == 0 && wq && p.cp_v != p.cp_g;
#define DG_SCA(NN, FF, HH) k_scalar_assemble<NN, FF, HH><<<grid, TPB, 0, st>>>(g, p, mode, phi, rho, cp, kc, D, mdot, u0, u1, u2, alpha_new, pinv, amb, Dg, c0, c1, c2, rhs, wq)
  if (hd) {
    if (nact(g) == 3) { if (g.fib) DG_SCA(3, true, true); else DG_SCA(3, false, true); }
    else { if (g.fib) DG_SCA(2, true, true); else DG_SCA(2, false, true); }
  } else {
    if (nact(g) == 3) { if (g.fib) DG_SCA(3, true, false); else DG_SCA(3, false, false); }
    else { if (g.fib) DG_SCA(2, true, false); else DG_SCA(2, false, false); }
  }
#undef DG_SCA
}

void L_mom_assemble(cudaStream_t st, int grid, Geo g, Phys p, int c, const double* u0, const double* u1, const double* u2, const double* rho, const double* mu, const double* pr, const double* alpha, const double* xi, double* Dg, double* c0, double* c1, double* c2, double* rhs, const Shadow32*) {
  ++g_launches;
#define DG_MOM(CC, NN, FF) k_mom_assemble<CC, NN, FF><<<grid, TPB, 0, st>>>(g, p, u0, u1, u2, rho, mu, pr, alpha, xi, Dg, c0, c1, c2, rhs)
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

void L_mom_scatter(cudaStream_t st, int grid, Geo g, Phys p, int c, const double* x, double* us) {
  ++g_launches;
  if (c == 0) k_mom_scatter<0><<<grid, TPB, 0, st>>>(g, p, x, us);
  else if (c == 1) k_mom_scatter<1><<<grid, TPB, 0, st>>>(g, p, x, us);
  else k_mom_scatter<2><<<grid, TPB, 0, st>>>(g, p, x, us);
}

void L_poisson_assemble(cudaStream_t st, int grid, Geo g, Phys p, const double* mdot, const double* alpha, const double* rgo, const double* rgn, const double* u0, const double* u1, const double* u2, const double* us0, const double* us1, const double* us2, const double* rho, const double* T1, const double* T0, double* expand, double* S, double* Dg, double* c0, double* c1, double* c2, double* rhs, double* dp0) {
  ++g_launches;
  if (nact(g) == 3) k_poisson_assemble<3><<<grid, TPB, 0, st>>>(g, p, mdot, alpha, rgo, rgn, u0, u1, u2, us0, us1, us2, rho, T1, T0, expand, S, Dg, c0, c1, c2, rhs, dp0);
  else k_poisson_assemble<2><<<grid, TPB, 0, st>>>(g, p, mdot, alpha, rgo, rgn, u0, u1, u2, us0, us1, us2, rho, T1, T0, expand, S, Dg, c0, c1, c2, rhs, dp0);
}

void L_correct(cudaStream_t st, int grid, Geo g, Phys p, int c, const double* us, const double* dp, const double* rho, double* u) {
  ++g_launches;
  if (c == 0) k_correct<0><<<grid, TPB, 0, st>>>(g, p, us, dp, rho, u);
  else if (c == 1) k_correct<1><<<grid, TPB, 0, st>>>(g, p, us, dp, rho, u);
  else k_correct<2><<<grid, TPB, 0, st>>>(g, p, us, dp, rho, u);
}

void L_correct_all(cudaStream_t st, Geo g, Phys p, double* const us[3], const double* dp, const double* rho,
                   double* const u[3], double* pr) {
  CorrectArgs a;
  const int na = nact(g);
  int b = 0;
  for (int c = 0; c < 3; ++c) {
    a.b[c] = b;
    a.us[c] = us[c];
    a.u[c] = u[c];
    if (c < na) b += lin_grid(nfaces(g, c));
  }
  a.b[3] = b;
  a.dp = dp;
  a.rho = rho;
  a.pr = pr;
  ++g_launches;
  k_correct_all<<<b + lin_grid(g.N), TPB, 0, st>>>(g, p, a);
}

void L_diag(cudaStream_t st, int grid, Geo g, Phys p, const double* alpha, const double* T, const double* mdot, const double* omega, const double* rhoG, const double* u0, const double* u1, const double* u2, double* psum, double* pmax, unsigned* flags) {
  ++g_launches;
  if (nact(g) == 3) k_diag<3><<<grid, TPB, 0, st>>>(g, p, alpha, T, mdot, omega, rhoG, u0, u1, u2, psum, pmax, flags);
  else k_diag<2><<<grid, TPB, 0, st>>>(g, p, alpha, T, mdot, omega, rhoG, u0, u1, u2, psum, pmax, flags);
}

void L_faces_to_box(cudaStream_t st, int grid, const Geo& g, int c, const double* u, double* x, double* uh,
                    const double* scal) {
  ++g_launches;
  if (c == 0) k_faces_to_box<0><<<grid, TPB, 0, st>>>(g, u, x, uh, scal);
  else if (c == 1) k_faces_to_box<1><<<grid, TPB, 0, st>>>(g, u, x, uh, scal);
  else k_faces_to_box<2><<<grid, TPB, 0, st>>>(g, u, x, uh, scal);
}

}  // namespace dg
