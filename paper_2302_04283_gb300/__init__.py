"""GB300 finite-solid-angle GR radiation: Python binding of librad.so.

Argument marshalling only.  Every step of the computation runs in the CUDA
library behind the C ABI declared in include/rad.h; this module converts
torch tensors to device pointers, numpy arrays to host pointers, checks
status codes and raises RadError with the library's message.  It never
computes a result itself, and it refuses to run when librad.so is missing.

Names match the C entry points: rad_create, rad_destroy, rad_init_angles,
rad_init_angles_latlong, rad_get_angles, rad_set_metric, rad_cfl_dt, rad_step, rad_moments,
rad_step_adjoint, rad_loss_outer, rad_check, rad_opts_default.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librad.so")

RAD_OK, RAD_EINVAL, RAD_ENOMEM, RAD_ECUDA, RAD_ENOCONV, RAD_ENONFINITE, RAD_ESTATE, RAD_EUNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6, -7
RAD_MINK_CART, RAD_MINK_SPH, RAD_KS_SPH = 0, 1, 2
RAD_BC_PERIODIC, RAD_BC_OUTFLOW, RAD_BC_POLAR, RAD_BC_HALO = 0, 1, 2, 3
RAD_F64, RAD_F32 = 0, 1
RAD_RECON_DC, RAD_RECON_PLM, RAD_RECON_PPM, RAD_RECON_MAPR = 0, 1, 2, 3
RAD_COUPLE_THERMAL, RAD_COUPLE_EMISSIVITY, RAD_COUPLE_NONE = 0, 1, 2
RAD_FRAME_TETRAD, RAD_FRAME_COORD, RAD_FRAME_FLUID = 0, 1, 2
RAD_MOM_SIMT, RAD_MOM_BF16X3 = 0, 1

KIND = {"mink_cart": RAD_MINK_CART, "mink_sph": RAD_MINK_SPH, "ks_sph": RAD_KS_SPH}
BC = {"periodic": RAD_BC_PERIODIC, "outflow": RAD_BC_OUTFLOW, "polar": RAD_BC_POLAR, "halo": RAD_BC_HALO}

_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


class rad_metric(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("spin", ctypes.c_double)]


class rad_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 3), ("xf", _dp * 3),
                ("bc_lo", ctypes.c_int * 3), ("bc_hi", ctypes.c_int * 3)]


class rad_gas(ctypes.Structure):
    _fields_ = [("rho", _vp), ("u", _vp), ("alpha_a", _vp), ("alpha_s", _vp), ("eta", _vp), ("T", _vp)]


class rad_host_item(ctypes.Structure):
    _fields_ = [("I", _vp), ("rho", _vp), ("u", _vp), ("alpha_a", _vp), ("alpha_s", _vp), ("eta", _vp),
                ("T", _vp), ("R", _vp), ("I_out", _vp)]


class rad_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("recon", ctypes.c_int), ("coupling", ctypes.c_int),
                ("n0crit", ctypes.c_double), ("zero_guard", ctypes.c_int), ("a_rad", ctypes.c_double),
                ("gamma", ctypes.c_double), ("tau_const", ctypes.c_double), ("rad_dom", ctypes.c_int),
                ("recon_ang", ctypes.c_int)]


class RadError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"rad status {status}: {msg}")
        self.status = status


_LIB = None


def lib():
    """Load librad.so (raises if it has not been built: there is no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with python -m paper_2302_04283_gb300.build")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    sig = {
        "rad_create": ([P(_vp), _vp], ctypes.c_int),
        "rad_destroy": ([_vp], None),
        "rad_last_error": ([_vp], ctypes.c_char_p),
        "rad_opts_default": ([P(rad_opts)], None),
        "rad_init_angles": ([_vp, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int)], ctypes.c_int),
        "rad_init_angles_latlong": ([_vp, ctypes.c_int, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int)],
                                    ctypes.c_int),
        "rad_get_angles": ([_vp, _vp, _vp, _vp], ctypes.c_int),
        "rad_set_metric": ([_vp, P(rad_metric), P(rad_grid)], ctypes.c_int),
        "rad_cfl_dt": ([_vp, ctypes.c_double, P(ctypes.c_double)], ctypes.c_int),
        "rad_step": ([_vp, _vp, P(rad_gas), ctypes.c_double, P(rad_opts), _vp], ctypes.c_int),
        "rad_step_noalloc": ([_vp, _vp, P(rad_gas), ctypes.c_double, P(rad_opts), _vp], ctypes.c_int),
        "rad_moments": ([_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, P(rad_gas), _vp], ctypes.c_int),
        "rad_step_adjoint": ([_vp, _vp, P(rad_gas), ctypes.c_double, P(rad_opts), _vp, _vp, _vp, _vp, _vp, _vp,
                              _vp], ctypes.c_int),
        "rad_loss_outer": ([_vp, _vp, ctypes.c_int, _vp, _vp], ctypes.c_int),
        "rad_step_host": ([_vp, ctypes.c_int, P(rad_host_item), ctypes.c_double, P(rad_opts), ctypes.c_int,
                           ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "rad_check": ([_vp], ctypes.c_int),
        "rad_selftest_wait": ([_vp, ctypes.c_double], ctypes.c_int),
        "rad_fp64_fma_rate": ([ctypes.c_double, P(ctypes.c_double)], ctypes.c_int),
        "rad_step_stage": ([_vp, ctypes.c_int, _vp, P(rad_gas), ctypes.c_double, P(rad_opts), _vp, _vp],
                           ctypes.c_int),
        "rad_halo_pack": ([_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp], ctypes.c_int),
        "rad_set_groups": ([_vp, ctypes.c_int, P(ctypes.c_double)], ctypes.c_int),
        "rad_gas_update": ([_vp, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_double], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _LIB = L
    return L


def _ptr(t):
    """Device (or host) address of a torch tensor, None -> NULL."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensors passed to librad must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _check(ctx, st):
    if st != RAD_OK:
        msg = lib().rad_last_error(ctx)
        raise RadError(st, msg.decode() if msg else "")


def rad_create(stream=None):
    """New context bound to a CUDA stream (torch.cuda.Stream or raw handle)."""
    h = ctypes.c_void_p()
    raw = getattr(stream, "cuda_stream", stream)
    st = lib().rad_create(ctypes.byref(h), ctypes.c_void_p(raw) if raw else None)
    if st != RAD_OK:
        raise RadError(st, "rad_create failed")
    return h


def rad_destroy(ctx):
    lib().rad_destroy(ctx)


def rad_opts_default(**kw):
    o = rad_opts()
    lib().rad_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def rad_init_angles(ctx, level):
    na, nap = ctypes.c_int(), ctypes.c_int()
    _check(ctx, lib().rad_init_angles(ctx, int(level), ctypes.byref(na), ctypes.byref(nap)))
    return na.value, nap.value


def rad_init_angles_latlong(ctx, n_zeta, n_psi):
    na, nap = ctypes.c_int(), ctypes.c_int()
    _check(ctx, lib().rad_init_angles_latlong(ctx, int(n_zeta), int(n_psi), ctypes.byref(na), ctypes.byref(nap)))
    return na.value, nap.value


def rad_get_angles(ctx, n_ang):
    d = np.zeros((n_ang, 3))
    w = np.zeros(n_ang)
    nb = np.zeros((n_ang, 6), dtype=np.int32)
    _check(ctx, lib().rad_get_angles(ctx, d.ctypes.data, w.ctypes.data, nb.ctypes.data))
    return d, w, nb


def rad_set_metric(ctx, kind, spin, ndim, xf, bc):
    """kind: 'mink_cart' | 'mink_sph' | 'ks_sph'; xf: three face arrays; bc: ((lo, hi),) * 3."""
    xs = [np.ascontiguousarray(np.asarray(x, dtype=np.float64)) for x in xf]
    g = rad_grid()
    g.ndim = ndim
    for d in range(3):
        g.n[d] = len(xs[d]) - 1
        g.xf[d] = xs[d].ctypes.data_as(_dp)
        g.bc_lo[d] = BC[bc[d][0]] if isinstance(bc[d][0], str) else bc[d][0]
        g.bc_hi[d] = BC[bc[d][1]] if isinstance(bc[d][1], str) else bc[d][1]
    m = rad_metric(KIND[kind] if isinstance(kind, str) else kind, float(spin))
    _check(ctx, lib().rad_set_metric(ctx, ctypes.byref(m), ctypes.byref(g)))


def rad_cfl_dt(ctx, cfl):
    dt = ctypes.c_double()
    _check(ctx, lib().rad_cfl_dt(ctx, float(cfl), ctypes.byref(dt)))
    return dt.value


def _gas(gas):
    g = rad_gas()
    if gas is None:
        return g
    for k in ("rho", "u", "alpha_a", "alpha_s", "eta", "T"):
        setattr(g, k, _ptr(gas.get(k)))
    return g


def rad_step(ctx, I, gas, dt, opts, gas_src=None):
    g = _gas(gas)
    _check(ctx, lib().rad_step(ctx, _ptr(I), ctypes.byref(g), float(dt), ctypes.byref(opts), _ptr(gas_src)))


def rad_step_noalloc(ctx, I, gas, dt, opts, gas_src=None):
    """rad_step with its stage scratch in the library's static device array
    (no device allocation; see include/rad.h for the size limit)."""
    g = _gas(gas)
    _check(ctx, lib().rad_step_noalloc(ctx, _ptr(I), ctypes.byref(g), float(dt), ctypes.byref(opts),
                                       _ptr(gas_src)))


def rad_step_stage(ctx, stage, I, gas, dt, opts, gas_src=None, halo=None):
    """One RK2 stage of a block; halo: dict {(d, side): device tensor} of the
    ghost layers of the block's shared faces (rad_halo_pack layout)."""
    g = _gas(gas)
    arr = (ctypes.c_void_p * 6)()
    for (d, side), t in (halo or {}).items():
        arr[2 * d + side] = _ptr(t).value if t is not None else None
    _check(ctx, lib().rad_step_stage(ctx, int(stage), _ptr(I), ctypes.byref(g), float(dt), ctypes.byref(opts),
                                     _ptr(gas_src), arr))


def rad_gas_update(ctx, rho, u, T, src, gamma=5.0 / 3.0):
    """Apply the step's gas source (src: [.., 4] or [n_groups, .., 4]) to the
    gas state (rho, u, T) the step started from, in place."""
    per = rho.numel() * 4
    if src.numel() % per:
        raise ValueError("src must hold whole [cell][4] arrays")
    _check(ctx, lib().rad_gas_update(ctx, _ptr(rho), _ptr(u), _ptr(T), _ptr(src), src.numel() // per,
                                     float(gamma)))


def rad_set_groups(ctx, nu_edges):
    """Multigroup transport with the given frequency edges (n_groups + 1
    values, increasing, the last may be inf); an empty list returns to gray."""
    e = [float(x) for x in nu_edges]
    ng = max(0, len(e) - 1)
    arr = (ctypes.c_double * max(1, len(e)))(*e)
    _check(ctx, lib().rad_set_groups(ctx, ng, arr))


def rad_halo_pack(ctx, I, precision, dim, side, buf):
    """Pack the 3 layers next to face (dim, side) of I (None: the context's
    stage-1 result) into buf."""
    _check(ctx, lib().rad_halo_pack(ctx, _ptr(I), int(precision), int(dim), int(side), _ptr(buf)))


def rad_step_host(ctx, items, dt, opts, nsteps, frame, method):
    """items: list of dicts of host (CPU, ideally pinned) tensors with keys
    I, rho, u, alpha_a, alpha_s, eta (or None), T (in/out), R (out) and
    optionally I_out.  Copies in, steps, takes the moments and copies back,
    overlapping the copies of neighbouring items with each item's steps."""
    arr = (rad_host_item * max(1, len(items)))()
    for n, it in enumerate(items):
        for k in ("I", "rho", "u", "alpha_a", "alpha_s", "T", "R"):
            if it[k].is_cuda:
                raise ValueError("rad_step_host takes host tensors")
        a = arr[n]
        for k in ("I", "rho", "u", "alpha_a", "alpha_s", "eta", "T", "R", "I_out"):
            setattr(a, k, _ptr(it.get(k)))
    _check(ctx, lib().rad_step_host(ctx, len(items), arr, float(dt), ctypes.byref(opts), int(nsteps), int(frame),
                                    int(method)))


def rad_moments(ctx, I, precision, frame, method, gas, R):
    g = _gas(gas)
    _check(ctx, lib().rad_moments(ctx, _ptr(I), precision, frame, method, ctypes.byref(g), _ptr(R)))


def rad_step_adjoint(ctx, I_n, gas, dt, opts, lam_np1, lam_n, lamT_np1, lamT_n, g_alpha_a, g_alpha_s,
                     g_eta=None):
    """lamT_np1 / lamT_n: adjoint of the gas temperature after / before the
    step (FP64 [k][j][i] device tensors, or None)."""
    g = _gas(gas)
    _check(ctx, lib().rad_step_adjoint(ctx, _ptr(I_n), ctypes.byref(g), float(dt), ctypes.byref(opts),
                                       _ptr(lam_np1), _ptr(lam_n), _ptr(lamT_np1), _ptr(lamT_n),
                                       _ptr(g_alpha_a), _ptr(g_alpha_s), _ptr(g_eta)))


def rad_loss_outer(ctx, I, precision, L_dev, dL_dI=None):
    _check(ctx, lib().rad_loss_outer(ctx, _ptr(I), precision, _ptr(L_dev), _ptr(dL_dI)))


def rad_check(ctx):
    _check(ctx, lib().rad_check(ctx))


def rad_selftest_wait(ctx, seconds):
    _check(ctx, lib().rad_selftest_wait(ctx, float(seconds)))


def rad_fp64_fma_rate(seconds=3.0):
    """Measured FP64 FMA rate of the current GPU in TFLOP/s."""
    out = ctypes.c_double()
    st = lib().rad_fp64_fma_rate(float(seconds), ctypes.byref(out))
    if st != RAD_OK:
        raise RadError(st, "rad_fp64_fma_rate failed")
    return out.value


def rad_last_error(ctx):
    msg = lib().rad_last_error(ctx)
    return msg.decode() if msg else ""
