"""Synthetic workloads: plain parameter dictionaries and seeded generators.

This module holds no arithmetic of the method.  It only names the cases (grid,
domain, operating conditions, time step) that the tests and the benchmark feed,
unchanged, to both the CUDA library and the CPU oracle.

Constants are round heptane / nitrogen-like values (the paper's property
libraries are not available): liquid rho 684, cp 2250, k 0.12, mu 3.9e-4,
D 1e-9; gas M 0.028013, cp 1100 (fuel vapour the same), k 0.055, mu 3.5e-5,
D 5e-5 m2/s at 1 bar; fuel M 0.100204, Tb 371.6 K, L 3.17e5 J/kg.  The case
shapes (D0 0.5-1.5 mm, ambient 300-1000 K, 1-20 bar, 0.7-1 m/s inflow) follow
the paper's case tables (Tables table1Dcases, tableGravityCases,
tableForcedCases).
"""
import copy

GEOM_AXISYM = 0
GEOM_CART3D = 1

# physics_mask bits: which stages of the segregated step are active
PHYS_EVAP = 1       # evaporation flux + alpha source (Sec. 2.4, Eq. alphasource)
PHYS_ENERGY = 2     # energy equation (Eq. Teqn)
PHYS_SPECIES = 4    # species equation (Eq. speciesequation)
PHYS_FLOW = 8       # momentum predictor + projection + alpha advection
PHYS_ALL = 15

BASE = dict(
    geom=GEOM_AXISYM, n=(64, 128, 1), L=(4e-3, 8e-3, 0.0), xc=(0.0, 4e-3, 0.0),
    D0=1e-3, T_drop=300.0, T_amb=773.0, P=1.0e5, g=(0.0, 0.0, 0.0), u_inflow=0.0,
    bc_mode=0, eq_model=0,
    Tb=371.6, Lv=3.17e5, M_l=0.100204, rho_l=684.0, cp_l=2250.0, k_l=0.12, mu_l=3.9e-4, D_l=1e-9,
    M_g=0.028013, cp_g=1100.0, cp_v=1100.0, k_g=0.055, mu_g=3.5e-5, D_g=5e-5,
    Tc=540.0, Pc=27.4e5, omega_ac=0.35, Tc_g=126.2, Pc_g=33.9e5, omega_g=0.037, kij=0.0,
    xi0=1.0, fiber_radius=5e-5, fiber=0,
    dt=1e-5, precision=0,
    cg_rtol=1e-12, cg_maxit=400, helm_rtol=1e-13, helm_maxit=400,
    seed=20050286, T_perturb=0.0,
    const_props_check=0, physics_mask=PHYS_ALL, C_alpha=4.0,
    mg_tile=(0, 0), wait_limit=0, solver_select=0, co_max=0.0, adv_scheme=0, drho_l_dT=0.0,
)


def make(**over):
    """A config dict: BASE with the given fields replaced."""
    cfg = copy.deepcopy(BASE)
    for k, v in over.items():
        if k not in cfg:
            raise KeyError(f"unknown config field {k}")
        cfg[k] = v
    return cfg


def cfg1_axisym_64x128(**over):
    """2D axisymmetric 64x128 over 4 x 8 mm, D0 = 1 mm on the axis, zero
    gravity, Raoult + Clausius-Clapeyron, 773 K, 1 bar, FP64, dt 1e-5 s."""
    return make(**over)


def cfg1_d2law(**over):
    """Constant-property microgravity check of the d2 law on the 64x128 grid:
    rho_G frozen at p M_g/(R T_amb), energy off, T = T_drop everywhere, initial
    vapour from the quasi-steady spherical Stefan profile.  dt 1e-4 s (the
    Stefan velocity stays below 0.04 m/s: Courant number < 0.07 at 62.5 um),
    so that a few hundred steps run well past the transient r_s^2/D = 5 ms.
    Interface compression C_alpha = 4 (the default of every case: at C_alpha = 1
    the outward Stefan flow carries liquid into the first gas cells over tens of
    milliseconds)."""
    base = dict(const_props_check=1, physics_mask=PHYS_EVAP | PHYS_SPECIES | PHYS_FLOW, dt=1e-4, C_alpha=4.0)
    base.update(over)
    return make(**base)


def cfg2_axisym_256x512(**over):
    """2D axisymmetric 256x512 over 4 x 8 mm, normal gravity, droplet held by
    the centripetal force, natural convection, 773 K, 1 bar, dt 5e-6 s."""
    base = dict(n=(256, 512, 1), g=(0.0, -9.81, 0.0), dt=5e-6, precision=1, cg_rtol=1e-8, helm_rtol=1e-8)
    base.update(over)
    return make(**base)


def cfg3_cart3d(nc=256, **over):
    """3D Cartesian nc^3 over a 4 mm cube, inflow 1 m/s at 773 K along +z,
    20 bar, Peng-Robinson equilibrium, D0 = 0.8 mm, 1 % seeded perturbation of
    the initial temperature, dt 2e-6 s."""
    base = dict(geom=GEOM_CART3D, n=(nc, nc, nc), L=(4e-3, 4e-3, 4e-3), xc=(2e-3, 2e-3, 2e-3),
                D0=0.8e-3, P=20e5, g=(0.0, 0.0, -9.81), u_inflow=1.0, bc_mode=1, eq_model=1,
                dt=2e-6, T_perturb=0.01, precision=1, cg_rtol=1e-8, helm_rtol=1e-8)
    base.update(over)
    return make(**base)


def cfg5_axisym_128x256(**over):
    """2D axisymmetric 128x256 over 4 x 8 mm, normal gravity, D0 = 1 mm, FP64."""
    base = dict(n=(128, 256, 1), g=(0.0, -9.81, 0.0))
    base.update(over)
    return make(**base)


def splitmix64(x):
    """SplitMix64 output for a 64-bit counter x (Steele, Lea & Flood 2014)."""
    m = (1 << 64) - 1
    z = (x + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def cfg4_batch(n_drop=64, seed=20050286, nr_choices=(64, 96, 128, 160, 192, 224, 256)):
    """Batch of axisymmetric droplets with seed-drawn grids and conditions:
    N_r uniform over nr_choices, N_z = 2 N_r, domain 4 D0 x 8 D0, D0 in
    [0.5, 1.5] mm, T_amb in [500, 1000] K, p in [1, 20] bar, gravity on,
    dt scaled with the cell size (1e-5 s at 62.5 um)."""
    out = []
    ctr = seed
    def u01():
        nonlocal ctr
        ctr += 1
        return (splitmix64(ctr) >> 11) * (1.0 / (1 << 53))
    for _ in range(n_drop):
        nr = nr_choices[min(int(u01() * len(nr_choices)), len(nr_choices) - 1)]
        d0 = 0.5e-3 + 1.0e-3 * u01()
        tamb = 500.0 + 500.0 * u01()
        p = 1e5 + 19e5 * u01()
        L0, L1 = 4 * d0, 8 * d0
        dx = L0 / nr
        out.append(make(n=(nr, 2 * nr, 1), L=(L0, L1, 0.0), xc=(0.0, 0.5 * L1, 0.0), D0=d0,
                        T_amb=tamb, P=p, g=(0.0, -9.81, 0.0), dt=1e-5 * dx / 62.5e-6,
                        precision=1, cg_rtol=1e-8, helm_rtol=1e-8))
    return out


def n_cells(cfg):
    n = cfg["n"]
    return n[0] * n[1] * n[2]
