"""Python binding of the droplet C ABI (include/droplet.h).

Argument marshalling only: every stage of the step runs in the CUDA library
libdroplet.so.  The module-level functions carry the C names (droplet_init,
droplet_step, droplet_diag, ...); the Droplet class wraps one context.
PyTorch supplies the CUDA stream (torch.cuda.current_stream()).

There is no CPU fallback: if libdroplet.so is missing or cannot be loaded the
import of the library raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libdroplet.so")

_c_int, _c_dbl = ctypes.c_int, ctypes.c_double


class DropletConfig(ctypes.Structure):
    _fields_ = [
        ("geom", _c_int), ("n", _c_int * 3), ("L", _c_dbl * 3), ("xc", _c_dbl * 3),
        ("D0", _c_dbl), ("T_drop", _c_dbl), ("T_amb", _c_dbl), ("P", _c_dbl), ("g", _c_dbl * 3), ("u_inflow", _c_dbl),
        ("bc_mode", _c_int), ("eq_model", _c_int),
        ("Tb", _c_dbl), ("Lv", _c_dbl), ("M_l", _c_dbl), ("rho_l", _c_dbl), ("cp_l", _c_dbl), ("k_l", _c_dbl),
        ("mu_l", _c_dbl), ("D_l", _c_dbl),
        ("M_g", _c_dbl), ("cp_g", _c_dbl), ("cp_v", _c_dbl), ("k_g", _c_dbl), ("mu_g", _c_dbl), ("D_g", _c_dbl),
        ("Tc", _c_dbl), ("Pc", _c_dbl), ("omega_ac", _c_dbl), ("Tc_g", _c_dbl), ("Pc_g", _c_dbl), ("omega_g", _c_dbl),
        ("kij", _c_dbl),
        ("xi0", _c_dbl), ("fiber_radius", _c_dbl),
        ("dt", _c_dbl), ("precision", _c_int),
        ("cg_rtol", _c_dbl), ("cg_maxit", _c_int), ("helm_rtol", _c_dbl), ("helm_maxit", _c_int),
        ("seed", ctypes.c_ulonglong), ("T_perturb", _c_dbl),
        ("const_props_check", _c_int), ("physics_mask", _c_int), ("C_alpha", _c_dbl),
        ("mg_tile", _c_int * 2), ("wait_limit", _c_int), ("solver_select", _c_int), ("co_max", _c_dbl),
        ("adv_scheme", _c_int), ("drho_l_dT", _c_dbl), ("fiber", _c_int),
    ]


class DropletDiag(ctypes.Structure):
    _fields_ = [
        ("t", _c_dbl), ("step", ctypes.c_longlong), ("V_l", _c_dbl), ("d_eq", _c_dbl), ("d2", _c_dbl),
        ("mdot_tot", _c_dbl), ("K_norm", _c_dbl), ("T_s_mean", _c_dbl), ("M_liq", _c_dbl), ("M_vap", _c_dbl),
        ("vap_out_cum", _c_dbl), ("max_u", _c_dbl), ("alpha_min", _c_dbl), ("alpha_max", _c_dbl),
        ("clip_mass", _c_dbl), ("its_p", _c_int), ("its_T", _c_int), ("its_w", _c_int), ("its_u", _c_int),
        ("res_p", _c_dbl), ("flags", ctypes.c_uint),
    ]


FIELDS = dict(alpha=0, T=1, omega=2, p=3, rhoG=4, u0=5, u1=6, u2=7, mdot=8, mraw=9, alpha_star=10, dp=11, S=12,
              ustar0=13, ustar1=14, ustar2=15, rhoG_old=16, expand=18)

EXPORTS = ["droplet_init", "droplet_step", "droplet_diag", "droplet_field_size", "droplet_get_field",
           "droplet_set_field", "droplet_sync", "droplet_free", "droplet_strerror", "droplet_profile",
           "droplet_profile_read", "droplet_launch_count", "droplet_box_solve", "droplet_box_solve_noalloc", "droplet_save", "droplet_load", "droplet_adjoint",
           "droplet_adjoint_vjp", "droplet_adjoint_check", "droplet_round_f32", "droplet_rcp_f64", "droplet_fp64_rate"]

NOALLOC_MAX_UNKNOWNS = 262144

# kernel classes timed by droplet_profile
KCLASS = dict(mg_smooth=0, spmv=1, update=2, mg_restrict=3, mg_prolong=4, mom_assemble=5, scalar_assemble=6,
              pcg_persist=7)

ERR_NOT_CONVERGED = -3
ERR_NONFINITE = -4
ERR_TIMEOUT = -8
FLAG_ADJ_NOT_FOUND = 8
FLAG_NONFINITE = 32

_lib = None


class DropletError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what}: {strerror(status)} ({status})")
        self.status = status


def load_library(path=LIBPATH):
    """Load libdroplet.so and declare the C signatures.  Raises when missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.droplet_init.argtypes = [ctypes.POINTER(DropletConfig), _c_int, P, ctypes.POINTER(P)]
    lib.droplet_step.argtypes = [P, _c_int]
    lib.droplet_diag.argtypes = [P, _c_int, ctypes.POINTER(DropletDiag)]
    lib.droplet_field_size.argtypes = [P, _c_int, _c_int, ctypes.POINTER(ctypes.c_size_t)]
    lib.droplet_get_field.argtypes = [P, _c_int, _c_int, ctypes.POINTER(_c_dbl), ctypes.c_size_t]
    lib.droplet_set_field.argtypes = [P, _c_int, _c_int, ctypes.POINTER(_c_dbl), ctypes.c_size_t]
    lib.droplet_sync.argtypes = [P]
    lib.droplet_free.argtypes = [P]
    lib.droplet_free.restype = None
    lib.droplet_profile.argtypes = [P, _c_int]
    lib.droplet_profile_read.argtypes = [P, _c_int, ctypes.POINTER(_c_dbl), ctypes.POINTER(ctypes.c_longlong),
                                         ctypes.POINTER(_c_dbl), ctypes.POINTER(_c_dbl)]
    lib.droplet_launch_count.argtypes = [P, ctypes.POINTER(ctypes.c_longlong)]
    BOX = [ctypes.POINTER(_c_int), P, P, P, P, P, P, _c_dbl, _c_int, P, ctypes.POINTER(_c_int), ctypes.POINTER(_c_dbl)]
    lib.droplet_box_solve.argtypes = BOX
    lib.droplet_box_solve_noalloc.argtypes = BOX
    D = ctypes.POINTER(_c_dbl)
    lib.droplet_adjoint.argtypes = [P, _c_int, _c_int, D, D, D, D, ctypes.c_size_t]
    lib.droplet_adjoint_vjp.argtypes = [P, D, D, ctypes.c_size_t, _c_dbl, D]
    lib.droplet_adjoint_check.argtypes = [P, D, _c_int]
    lib.droplet_round_f32.argtypes = [P, P, P, ctypes.c_size_t]
    lib.droplet_rcp_f64.argtypes = [P, P, ctypes.c_size_t]
    lib.droplet_fp64_rate.argtypes = [ctypes.POINTER(_c_dbl)]
    lib.droplet_save.argtypes = [P, ctypes.c_char_p]
    lib.droplet_load.argtypes = [P, ctypes.c_char_p]
    lib.droplet_strerror.argtypes = [_c_int]
    lib.droplet_strerror.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("droplet_free", "droplet_strerror"):
            getattr(lib, name).restype = _c_int
    _lib = lib
    return lib


def strerror(status):
    return load_library().droplet_strerror(int(status)).decode()


def make_config(cfg):
    """droplet_config from a plain dict (see workloads.BASE for the keys)."""
    c = DropletConfig()
    for name, typ in DropletConfig._fields_:
        v = cfg[name]
        if isinstance(v, (tuple, list)):
            arr = getattr(c, name)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(c, name, typ(v).value if typ is not ctypes.c_ulonglong else int(v))
    return c


# ------------------------------------------------------------ C-named wrappers

def droplet_init(cfg, stream=None):
    """Returns the context handle (int).  cfg: one config dict, or a list of them
    (a batch of independent droplets stepped together).  stream: a cudaStream_t
    as int, or None for torch's current stream on the current device."""
    lib = load_library()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    cfgs = cfg if isinstance(cfg, (list, tuple)) else [cfg]
    arr = (DropletConfig * len(cfgs))(*[make_config(x) for x in cfgs])
    h = ctypes.c_void_p()
    rc = lib.droplet_init(arr, len(cfgs), ctypes.c_void_p(stream), ctypes.byref(h))
    if rc:
        raise DropletError(rc, "droplet_init")
    return h.value


def droplet_step(h, n_steps=1):
    rc = load_library().droplet_step(ctypes.c_void_p(h), int(n_steps))
    if rc and rc not in (ERR_NOT_CONVERGED, ERR_TIMEOUT):   # the state advanced: status returned
        raise DropletError(rc, "droplet_step")
    return rc


def droplet_diag(h, droplet=0):
    d = DropletDiag()
    rc = load_library().droplet_diag(ctypes.c_void_p(h), int(droplet), ctypes.byref(d))
    if rc:
        raise DropletError(rc, "droplet_diag")
    return {name: getattr(d, name) for name, _ in DropletDiag._fields_}


def droplet_field_size(h, field, droplet=0):
    n = ctypes.c_size_t()
    rc = load_library().droplet_field_size(ctypes.c_void_p(h), droplet, FIELDS[field], ctypes.byref(n))
    if rc:
        raise DropletError(rc, "droplet_field_size")
    return n.value


def droplet_get_field(h, field, out=None, droplet=0):
    n = droplet_field_size(h, field, droplet)
    if out is None:
        out = np.empty(n, dtype=np.float64)
    assert out.dtype == np.float64 and out.flags.c_contiguous
    rc = load_library().droplet_get_field(ctypes.c_void_p(h), droplet, FIELDS[field],
                                          out.ctypes.data_as(ctypes.POINTER(_c_dbl)), out.size)
    if rc:
        raise DropletError(rc, "droplet_get_field")
    return out


def droplet_set_field(h, field, values, droplet=0):
    v = np.ascontiguousarray(values, dtype=np.float64).ravel()
    rc = load_library().droplet_set_field(ctypes.c_void_p(h), droplet, FIELDS[field],
                                          v.ctypes.data_as(ctypes.POINTER(_c_dbl)), v.size)
    if rc:
        raise DropletError(rc, "droplet_set_field")


def droplet_get_field_ptr(h, field, ptr, n, droplet=0):
    """Copy a field into caller memory at address ptr (n doubles), e.g. pinned host memory."""
    rc = load_library().droplet_get_field(ctypes.c_void_p(h), droplet, FIELDS[field],
                                          ctypes.cast(ctypes.c_void_p(ptr), ctypes.POINTER(_c_dbl)), n)
    if rc:
        raise DropletError(rc, "droplet_get_field")


def droplet_set_field_ptr(h, field, ptr, n, droplet=0):
    rc = load_library().droplet_set_field(ctypes.c_void_p(h), droplet, FIELDS[field],
                                          ctypes.cast(ctypes.c_void_p(ptr), ctypes.POINTER(_c_dbl)), n)
    if rc:
        raise DropletError(rc, "droplet_set_field")


def droplet_profile(h, enable):
    rc = load_library().droplet_profile(ctypes.c_void_p(h), int(enable))
    if rc:
        raise DropletError(rc, "droplet_profile")


def droplet_profile_read(h, kclass):
    """(ms_total, launches, algorithmic_bytes_total, binary64_instructions_total) of a kernel
    class since droplet_profile(h, 1)."""
    ms, n, b, f = _c_dbl(), ctypes.c_longlong(), _c_dbl(), _c_dbl()
    k = KCLASS[kclass] if isinstance(kclass, str) else int(kclass)
    rc = load_library().droplet_profile_read(ctypes.c_void_p(h), k, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b),
                                             ctypes.byref(f))
    if rc:
        raise DropletError(rc, "droplet_profile_read")
    return ms.value, n.value, b.value, f.value


def droplet_round_f32(x):
    """The device's integer-pipe binary64 -> binary32 rounding and its exact widening
    back, applied to a float64 numpy array: returns (float32 array, float64 array)."""
    import numpy as np
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty(x.size, dtype=np.float32)
    back = np.empty(x.size, dtype=np.float64)
    rc = load_library().droplet_round_f32(x.ctypes.data, out.ctypes.data, back.ctypes.data, x.size)
    if rc:
        raise DropletError(rc, "droplet_round_f32")
    return out, back


def droplet_rcp_f64(x):
    """The device's binary64 reciprocal (binary32 seed, two Newton-Raphson steps)
    applied to a float64 numpy array."""
    import numpy as np
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty(x.size, dtype=np.float64)
    rc = load_library().droplet_rcp_f64(x.ctypes.data, out.ctypes.data, x.size)
    if rc:
        raise DropletError(rc, "droplet_rcp_f64")
    return out


def droplet_launch_count(h):
    n = ctypes.c_longlong()
    rc = load_library().droplet_launch_count(ctypes.c_void_p(h), ctypes.byref(n))
    if rc:
        raise DropletError(rc, "droplet_launch_count")
    return n.value


def _box_call(fn, m, D, c0, c1, c2, b, x, rtol, maxit, stream):
    mm = (_c_int * 3)(*[int(v) for v in m])
    its, rel = _c_int(), _c_dbl()
    rc = fn(mm, ctypes.c_void_p(D), ctypes.c_void_p(c0), ctypes.c_void_p(c1),
            ctypes.c_void_p(c2) if c2 else None, ctypes.c_void_p(b), ctypes.c_void_p(x),
            float(rtol), int(maxit), ctypes.c_void_p(stream), ctypes.byref(its), ctypes.byref(rel))
    return rc, its.value, rel.value


def droplet_box_solve(m, D, c0, c1, c2, b, x, rtol, maxit, stream):
    """Device pointers (ints) of the box system; returns (status, iterations, relative residual)."""
    return _box_call(load_library().droplet_box_solve, m, D, c0, c1, c2, b, x, rtol, maxit, stream)


def droplet_box_solve_noalloc(m, D, c0, c1, c2, b, x, rtol, maxit, stream):
    """droplet_box_solve with the work vectors in the library's static device array
    (no device allocation; at most NOALLOC_MAX_UNKNOWNS unknowns; calls must not overlap)."""
    return _box_call(load_library().droplet_box_solve_noalloc, m, D, c0, c1, c2, b, x, rtol, maxit, stream)


def droplet_save(h, path):
    rc = load_library().droplet_save(ctypes.c_void_p(h), os.fsencode(path))
    if rc:
        raise DropletError(rc, "droplet_save")


def droplet_load(h, path):
    rc = load_library().droplet_load(ctypes.c_void_p(h), os.fsencode(path))
    if rc:
        raise DropletError(rc, "droplet_load")


def droplet_adjoint(h, n_steps, ckpt_every, gradients=True):
    """J (mean evaporation rate) and, if gradients, (dJ/dT_amb, dJ/dD_g, dJ/dT0 as a
    flat array).  The context must be at step 0, with physics_mask EVAP|ENERGY|SPECIES
    or all four terms (the adjoint with flow)."""
    J = _c_dbl()
    if not gradients:
        rc = load_library().droplet_adjoint(ctypes.c_void_p(h), int(n_steps), int(ckpt_every), ctypes.byref(J),
                                            None, None, None, 0)
        if rc and rc != ERR_NOT_CONVERGED:
            raise DropletError(rc, "droplet_adjoint")
        return J.value
    n = droplet_field_size(h, "T")
    gT0 = np.empty(n, dtype=np.float64)
    gTa, gDg = _c_dbl(), _c_dbl()
    rc = load_library().droplet_adjoint(ctypes.c_void_p(h), int(n_steps), int(ckpt_every), ctypes.byref(J),
                                        ctypes.byref(gTa), ctypes.byref(gDg),
                                        gT0.ctypes.data_as(ctypes.POINTER(_c_dbl)), n)
    if rc and rc != ERR_NOT_CONVERGED:
        raise DropletError(rc, "droplet_adjoint")
    return J.value, gTa.value, gDg.value, gT0


STATE_FIELDS = ("alpha", "T", "omega", "p")


def state_size(h):
    """Length of the packed state of the flow adjoint: alpha, T, omega, p, then the face
    velocities of each active direction."""
    n = 4 * droplet_field_size(h, "T")
    for a in range(3):
        try:
            n += droplet_field_size(h, "u%d" % a)
        except DropletError:
            break
    return n


def droplet_adjoint_vjp(h, lam_next, mdot_weight=0.0):
    """One step of the flow adjoint: (lam_prev, dpar) for the step from the current state,
    lam_next and lam_prev packed as state_size describes; dpar = (T_amb, D_g)."""
    lam_next = np.ascontiguousarray(lam_next, dtype=np.float64)
    out = np.empty_like(lam_next)
    dpar = np.zeros(2, dtype=np.float64)
    P = ctypes.POINTER(_c_dbl)
    rc = load_library().droplet_adjoint_vjp(ctypes.c_void_p(h), lam_next.ctypes.data_as(P), out.ctypes.data_as(P),
                                            lam_next.size, float(mdot_weight), dpar.ctypes.data_as(P))
    if rc and rc != ERR_NOT_CONVERGED:
        raise DropletError(rc, "droplet_adjoint_vjp")
    return out, dpar


CHECK_NAMES = ("FL", "AF", "aL", "Rp", "Rm", "alpha1", "mraw", "energy_D", "energy_rhs", "energy_c", "species_D",
               "species_rhs", "species_c", "mom_D", "mom_rhs", "mom_c", "p_D", "p_rhs", "p_c", "correct")


def droplet_adjoint_check(h):
    """Relative differences between the flow adjoint's stage formulas and the forward
    kernels over one step from the current state, by stage name."""
    rel = np.zeros(len(CHECK_NAMES), dtype=np.float64)
    rc = load_library().droplet_adjoint_check(ctypes.c_void_p(h), rel.ctypes.data_as(ctypes.POINTER(_c_dbl)),
                                              len(CHECK_NAMES))
    if rc and rc != ERR_NOT_CONVERGED:
        raise DropletError(rc, "droplet_adjoint_check")
    return dict(zip(CHECK_NAMES, rel.tolist()))


def droplet_fp64_rate():
    """Measured binary64 FMA throughput of the current device [TFLOP/s]."""
    v = _c_dbl()
    rc = load_library().droplet_fp64_rate(ctypes.byref(v))
    if rc:
        raise DropletError(rc, "droplet_fp64_rate")
    return v.value


def droplet_sync(h):
    rc = load_library().droplet_sync(ctypes.c_void_p(h))
    if rc:
        raise DropletError(rc, "droplet_sync")


def droplet_free(h):
    load_library().droplet_free(ctypes.c_void_p(h))


class Droplet:
    """A context of one droplet (cfg a dict) or of a batch (cfg a list of dicts)
    on the current CUDA device."""

    def __init__(self, cfg, stream=None):
        self.cfg = cfg
        self.n = len(cfg) if isinstance(cfg, (list, tuple)) else 1
        self.h = droplet_init(cfg, stream)
        self.last_status = 0

    def step(self, n=1):
        self.last_status = droplet_step(self.h, n)
        return self.last_status

    def diag(self, droplet=0):
        return droplet_diag(self.h, droplet)

    def get(self, field, droplet=0):
        return droplet_get_field(self.h, field, droplet=droplet)

    def set(self, field, values, droplet=0):
        droplet_set_field(self.h, field, values, droplet=droplet)

    def sync(self):
        droplet_sync(self.h)

    def save(self, path):
        droplet_save(self.h, path)

    def load(self, path):
        droplet_load(self.h, path)

    def close(self):
        if self.h:
            droplet_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def evaporation_rate_function():
    """torch.autograd.Function J(T_amb, D_g, dT0): mean evaporation rate over
    n_steps of the step (with or without flow, as cfg's physics mask says), from the
    initial state with T0 = profile(T_amb) + dT0.  Backward returns the hand-written
    adjoint's gradient, computed (with checkpointing) when the forward runs."""
    import torch

    class EvaporationRate(torch.autograd.Function):
        @staticmethod
        def forward(ctx, T_amb, D_g, dT0, cfg, n_steps, ckpt_every):
            c = dict(cfg, T_amb=float(T_amb), D_g=float(D_g))
            sim = Droplet(c)
            if dT0 is not None:
                T0 = sim.get("T") + dT0.detach().cpu().numpy().ravel()
                sim.set("T", T0)
            J, gTa, gDg, gT0 = droplet_adjoint(sim.h, n_steps, ckpt_every, gradients=True)
            sim.close()
            ctx.save_for_backward(torch.tensor(gTa, dtype=torch.float64), torch.tensor(gDg, dtype=torch.float64),
                                  torch.from_numpy(gT0))
            return torch.tensor(J, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gJ):
            gTa, gDg, gT0 = ctx.saved_tensors
            return gJ * gTa, gJ * gDg, gJ * gT0, None, None, None

    return EvaporationRate
