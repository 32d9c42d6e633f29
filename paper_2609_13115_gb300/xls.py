"""Thin ctypes binding of libxls (include/xls.h): the same entry points, argument marshalling only.

Host arrays are numpy arrays (float64 / int32, C-contiguous); device arrays are torch CUDA
tensors (their data_ptr is passed with the on_device flag set).  Every call raises XlsError
with the library's message when the status is not XLS_OK.  There is no fallback: if the
shared library is missing the import-time loader raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int, c_size_t, c_uint64, c_void_p

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libxls.so")

XLS_OK, XLS_EINVAL, XLS_ENOMEM, XLS_ECUDA, XLS_ENOTSPD, XLS_ENOCONV, XLS_ETIMEOUT, XLS_ENONFINITE = range(8)
XLS_FP64, XLS_MIXED_BF16, XLS_MIXED_FP16 = 0, 1, 2
STATUS_NAMES = {0: "XLS_OK", 1: "XLS_EINVAL", 2: "XLS_ENOMEM", 3: "XLS_ECUDA", 4: "XLS_ENOTSPD",
                5: "XLS_ENOCONV", 6: "XLS_ETIMEOUT", 7: "XLS_ENONFINITE"}


class XlsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class XlsCell(ctypes.Structure):
    _fields_ = [("L", c_double * 3), ("n", c_int * 3)]


class XlsDC(ctypes.Structure):
    _fields_ = [("n_sub", c_int), ("core_lo", POINTER(c_int)), ("core_n", POINTER(c_int)),
                ("buf", POINTER(c_int)), ("n_states", POINTER(c_int))]


class XlsSpecies(ctypes.Structure):
    _fields_ = [("Zv", c_double), ("rc_loc", c_double), ("w_proj", c_double), ("r_cut", c_double),
                ("E_s", c_double), ("E_p", c_double)]


_SIGS = {
    "xls_grid_create": (c_int, [POINTER(XlsCell), POINTER(XlsDC), c_int, c_size_t, c_void_p, POINTER(c_void_p)]),
    "xls_grid_destroy": (c_int, [c_void_p]),
    "xls_hamiltonian_set": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p, c_void_p, c_int,
                                    POINTER(XlsSpecies)]),
    "xls_orbitals_set": (c_int, [c_void_p, c_int, c_void_p, c_int]),
    "xls_orbitals_random": (c_int, [c_void_p, c_uint64]),
    "xls_orbitals_get": (c_int, [c_void_p, c_int, c_void_p, c_int]),
    "xls_orbitals_set_f32": (c_int, [c_void_p, c_int, c_void_p, c_int]),
    "xls_autotune": (c_int, [c_void_p, c_int, c_void_p]),
    "xls_orbitals_get_f32": (c_int, [c_void_p, c_int, c_void_p, c_int]),
    "xls_chefsi_batch": (c_int, [c_void_p, c_int, c_int, c_void_p]),
    "xls_chefsi_stage": (c_int, [c_void_p, c_int, c_int, c_void_p]),
    "xls_hamiltonian_apply": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_int]),
    "xls_density": (c_int, [c_void_p, c_double, c_double, POINTER(c_double), c_void_p, c_int,
                            POINTER(c_double), POINTER(c_double)]),
    "xls_get_eigs": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "xls_get_subspace": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "xls_get_rotation": (c_int, [c_void_p, c_int, c_void_p]),
    "xls_get_eig_work": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "xls_wave_carry": (c_int, [c_void_p, c_int]),
    "xls_chefsi_wave": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p]),
    "xls_dos": (c_int, [c_void_p, c_void_p, c_int, c_double, c_void_p]),
    "xls_scf_cg_iterations": (c_int, [c_void_p, c_void_p]),
    "xls_wave_store_fp16": (c_int, [c_void_p, c_int]),
    "xls_get_bounds": (c_int, [c_void_p, c_void_p]),
    "xls_get_timings": (c_int, [c_void_p, c_void_p, POINTER(c_int)]),
    "xls_set_profiling": (c_int, [c_void_p, c_int]),
    "xls_set_graphs": (c_int, [c_void_p, c_int]),
    "xls_get_waves": (c_int, [c_void_p, POINTER(c_int), c_void_p]),
    "xls_fermi_partial": (c_int, [c_void_p, c_double, c_double, c_void_p]),
    "xls_selftest_wait": (c_int, [c_int, c_void_p]),
    "xls_orbitals_store_fp16": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "xls_orbitals_load_fp16": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "xls_fermi_histogram": (c_int, [c_void_p, c_double, c_double, c_int, c_void_p]),
    "xls_density_at": (c_int, [c_void_p, c_double, c_double, c_void_p, c_int, c_void_p]),
    "xls_mlp_create": (c_int, [c_void_p, c_int, c_void_p, POINTER(c_void_p)]),
    "xls_mlp_destroy": (c_int, [c_void_p]),
    "xls_mlp_get_params": (c_int, [c_void_p, c_void_p]),
    "xls_mlp_infer": (c_int, [c_void_p, c_void_p, ctypes.c_longlong, c_void_p, c_int]),
    "xls_mlp_loss_grad": (c_int, [c_void_p, c_void_p, c_void_p, ctypes.c_longlong, POINTER(c_double), c_void_p, c_int]),
    "xls_mlp_train_step": (c_int, [c_void_p, c_void_p, c_void_p, ctypes.c_longlong, c_double, POINTER(c_double), c_int]),
    "xls_descriptors": (c_int, [c_void_p, c_void_p, c_int]),
    "xls_learned_start": (c_int, [c_void_p, c_void_p, c_double, c_void_p, c_int]),
    "xls_scf_setup": (c_int, [c_void_p, c_double, c_double, c_int, c_int, c_double, c_double, c_int, c_int]),
    "xls_scf_step": (c_int, [c_void_p, c_void_p, c_int, POINTER(c_double), POINTER(c_double), POINTER(c_double)]),
    "xls_get_kernel_times": (c_int, [c_void_p, c_void_p, c_void_p]),
    "xls_gram_noalloc": (c_int, [c_void_p, c_void_p, ctypes.c_longlong, c_int, c_void_p, c_void_p, c_void_p]),
    "xls_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libxls.so (built by paper_2609_13115_gb300.build); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libxls.so not found at {path}: build it with paper_2609_13115_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> list:
    return list(_SIGS)


def _check(status: int):
    if status != XLS_OK:
        raise XlsError(status, load().xls_last_error().decode())


def _ptr(a):
    """(pointer, on_device) of a numpy array or a torch tensor; None -> (None, 0)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data_as(c_void_p), 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    raise TypeError(f"unsupported array type {type(a)}")


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32).ravel())


def xls_grid_create(L, n, core_lo, core_n, buf, n_states, precision=XLS_FP64, hbm_budget_bytes=0, stream=None):
    lib = load()
    cell = XlsCell((c_double * 3)(*[float(x) for x in L]), (c_int * 3)(*[int(x) for x in n]))
    arrs = [_i32(core_lo), _i32(core_n), _i32(buf), _i32(n_states)]
    dc = XlsDC(len(arrs[3]), *[a.ctypes.data_as(POINTER(c_int)) for a in arrs])
    h = c_void_p()
    _check(lib.xls_grid_create(byref(cell), byref(dc), int(precision), int(hbm_budget_bytes),
                               c_void_p(stream) if stream else None, byref(h)))
    return h


def xls_grid_destroy(g):
    _check(load().xls_grid_destroy(g))


def species_array(species) -> ctypes.Array:
    arr = (XlsSpecies * len(species))()
    for i, s in enumerate(species):
        arr[i] = XlsSpecies(s.Zv, s.rc_loc, s.w_proj, s.r_cut, s.E_s, s.E_p)
    return arr


def xls_hamiltonian_set(g, veff, pos, species_index, species):
    v = np.ascontiguousarray(veff, dtype=np.float64) if isinstance(veff, np.ndarray) else veff
    vp, vdev = _ptr(v)
    p = np.ascontiguousarray(pos, dtype=np.float64).ravel()
    s = _i32(species_index)
    sp = species_array(species)
    _check(load().xls_hamiltonian_set(g, vp, vdev, len(s), p.ctypes.data_as(c_void_p), s.ctypes.data_as(c_void_p),
                                      len(species), sp))


def xls_orbitals_set(g, sub, psi):
    a = np.ascontiguousarray(psi, dtype=np.float64) if isinstance(psi, np.ndarray) else psi
    p, dev = _ptr(a)
    _check(load().xls_orbitals_set(g, int(sub), p, dev))


def _require_f32(a):
    dt = a.dtype if isinstance(a, np.ndarray) else getattr(a, "dtype", None)
    if str(dt) not in ("float32", "torch.float32"):
        raise TypeError(f"FP32 orbital arrays must be float32, got {dt}")


def xls_orbitals_set_f32(g, sub, psi):
    a = np.ascontiguousarray(psi, dtype=np.float32) if isinstance(psi, np.ndarray) else psi
    _require_f32(a)
    p, dev = _ptr(a)
    _check(load().xls_orbitals_set_f32(g, int(sub), p, dev))


def xls_orbitals_get_f32(g, sub, out):
    _require_f32(out)
    p, dev = _ptr(out)
    _check(load().xls_orbitals_get_f32(g, int(sub), p, dev))
    return out


def xls_orbitals_random(g, seed):
    _check(load().xls_orbitals_random(g, int(seed)))


def xls_orbitals_get(g, sub, out):
    p, dev = _ptr(out)
    _check(load().xls_orbitals_get(g, int(sub), p, dev))
    return out


def xls_chefsi_batch(g, degree, n_passes, bounds=None):
    b = None if bounds is None else np.ascontiguousarray(bounds, dtype=np.float64).ravel()
    _check(load().xls_chefsi_batch(g, int(degree), int(n_passes), None if b is None else b.ctypes.data_as(c_void_p)))


def xls_autotune(g, reps=5):
    """Time the tunable launch configurations on the grid's data, keep the fastest; returns
    (cluster CTAs of the factorisations, Gram CTAs per SM aimed at, projection vectors per CTA),
    0 where not tuned."""
    out = np.zeros(3, dtype=np.int32)
    _check(load().xls_autotune(g, int(reps), out.ctypes.data_as(c_void_p)))
    return int(out[0]), int(out[1]), int(out[2])


def xls_chefsi_stage(g, stage, degree, bounds=None):
    b = None if bounds is None else np.ascontiguousarray(bounds, dtype=np.float64).ravel()
    _check(load().xls_chefsi_stage(g, int(stage), int(degree), None if b is None else b.ctypes.data_as(c_void_p)))


def xls_hamiltonian_apply(g, sub, x, y):
    xp, dev = _ptr(x)
    yp, dev2 = _ptr(y)
    if dev != dev2:
        raise ValueError("x and y must both be host or both be device arrays")
    k = x.shape[0] if x.ndim == 2 else 1
    _check(load().xls_hamiltonian_apply(g, int(sub), int(k), xp, yp, dev))
    return y


def xls_density(g, n_electrons, kT, rho_out=None):
    mu, eb, es = c_double(), c_double(), c_double()
    rp, dev = _ptr(rho_out)
    _check(load().xls_density(g, float(n_electrons), float(kT), byref(mu), rp, dev, byref(eb), byref(es)))
    return mu.value, eb.value, es.value


def xls_get_eigs(g, sub, n_states):
    lam = np.zeros(n_states)
    c = np.zeros(n_states)
    _check(load().xls_get_eigs(g, int(sub), lam.ctypes.data_as(c_void_p), c.ctypes.data_as(c_void_p)))
    return lam, c


def xls_get_eigs_into(g, sub, lam, c):
    """xls_get_eigs into caller-owned contiguous float64 arrays (no allocation per call)."""
    _check(load().xls_get_eigs(g, int(sub), lam.ctypes.data_as(c_void_p), c.ctypes.data_as(c_void_p)))


def xls_wave_store_fp16(g, on=True):
    _check(load().xls_wave_store_fp16(g, 1 if on else 0))


def xls_wave_carry(g, slots=-1):
    """Carry mode with `slots` subdomains per wave (-1: as many as the HBM budget allows; 0: off)."""
    _check(load().xls_wave_carry(g, int(slots)))


def xls_chefsi_wave(g, wave, degree, n_passes=1, bounds=None):
    b = None if bounds is None else np.ascontiguousarray(bounds, dtype=np.float64).ravel()
    _check(load().xls_chefsi_wave(g, int(wave), int(degree), int(n_passes),
                                  None if b is None else b.ctypes.data_as(c_void_p)))


def xls_scf_cg_iterations(g):
    it = ctypes.c_longlong(0)
    _check(load().xls_scf_cg_iterations(g, byref(it)))
    return int(it.value)


def xls_dos(g, energies, width):
    """Gaussian-broadened density of states (Eq. dos) at the given energies (Ha)."""
    e = np.ascontiguousarray(energies, dtype=np.float64).ravel()
    out = np.zeros_like(e)
    _check(load().xls_dos(g, e.ctypes.data_as(c_void_p), int(e.size), float(width), out.ctypes.data_as(c_void_p)))
    return out


def xls_get_subspace(g, sub, n_states):
    Ms = np.zeros((n_states, n_states))
    Hs = np.zeros((n_states, n_states))
    _check(load().xls_get_subspace(g, int(sub), Ms.ctypes.data_as(c_void_p), Hs.ctypes.data_as(c_void_p)))
    return Ms, Hs


def xls_get_rotation(g, sub, n_states):
    Y = np.zeros((n_states, n_states))
    _check(load().xls_get_rotation(g, int(sub), Y.ctypes.data_as(c_void_p)))
    return Y


def xls_get_eig_work(g, sub, n_states):
    """(L, A after tridiagonalisation, vecs[8, n]) of the last eigensolve of subdomain `sub`."""
    L = np.zeros((n_states, n_states))
    A = np.zeros((n_states, n_states))
    v = np.zeros(8 * n_states)
    _check(load().xls_get_eig_work(g, int(sub), L.ctypes.data_as(c_void_p), A.ctypes.data_as(c_void_p),
                                   v.ctypes.data_as(c_void_p)))
    return L, A, v.reshape(8, n_states)


def xls_get_bounds(g, n_sub):
    b = np.zeros(3 * n_sub)
    _check(load().xls_get_bounds(g, b.ctypes.data_as(c_void_p)))
    return b.reshape(n_sub, 3)


def xls_get_timings(g):
    ms = np.zeros(4)
    n = c_int()
    _check(load().xls_get_timings(g, ms.ctypes.data_as(c_void_p), byref(n)))
    return ms, n.value


def xls_set_profiling(g, on):
    _check(load().xls_set_profiling(g, int(bool(on))))


def xls_orbitals_store_fp16(g, sub, n_states, n_points):
    """(half values as uint16 array (n_states, n_points), exponents (n_states,))."""
    h = np.zeros((int(n_states), int(n_points)), dtype=np.uint16)
    e = np.zeros(int(n_states), dtype=np.int32)
    _check(load().xls_orbitals_store_fp16(g, int(sub), h.ctypes.data_as(c_void_p), e.ctypes.data_as(c_void_p)))
    return h, e


def xls_orbitals_load_fp16(g, sub, h, e):
    h = np.ascontiguousarray(h, dtype=np.uint16)
    e = np.ascontiguousarray(e, dtype=np.int32)
    _check(load().xls_orbitals_load_fp16(g, int(sub), h.ctypes.data_as(c_void_p), e.ctypes.data_as(c_void_p)))


def xls_selftest_wait(spin_limit=64, stream=None):
    _check(load().xls_selftest_wait(int(spin_limit), c_void_p(stream) if stream else None))


def xls_fermi_partial(g, mu, kT):
    out = np.zeros(4)
    _check(load().xls_fermi_partial(g, float(mu), float(kT), out.ctypes.data_as(c_void_p)))
    return out


def xls_fermi_histogram(g, lo, hi, n_bins):
    out = np.zeros(int(n_bins))
    _check(load().xls_fermi_histogram(g, float(lo), float(hi), int(n_bins), out.ctypes.data_as(c_void_p)))
    return out


def xls_density_at(g, mu, kT, rho=None):
    """Occupations at mu; fills rho (numpy, global grid) when given; returns [E_band, E_entropy, N_e]."""
    e3 = np.zeros(3)
    p = rho.ctypes.data_as(c_void_p) if rho is not None else None
    _check(load().xls_density_at(g, float(mu), float(kT), p, 0, e3.ctypes.data_as(c_void_p)))
    return e3


def xls_get_waves(g, n_sub):
    """(number of waves, first subdomain of each wave)."""
    n = c_int()
    first = np.zeros(max(1, n_sub), dtype=np.int32)
    _check(load().xls_get_waves(g, byref(n), first.ctypes.data_as(c_void_p)))
    return n.value, first[:n.value].tolist()


N_MLP_PARAMS = 10497


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(c_void_p)


def xls_mlp_create(params, stream=None):
    p = np.ascontiguousarray(params, dtype=np.float64)
    h = c_void_p()
    _check(load().xls_mlp_create(p.ctypes.data_as(c_void_p), int(p.size), c_void_p(stream) if stream else None,
                                 byref(h)))
    return h


def xls_mlp_destroy(m):
    _check(load().xls_mlp_destroy(m))


def xls_mlp_get_params(m):
    out = np.zeros(N_MLP_PARAMS)
    _check(load().xls_mlp_get_params(m, out.ctypes.data_as(c_void_p)))
    return out


def xls_mlp_infer(m, X):
    X, px = _f32(X)
    y = np.zeros(X.shape[0], dtype=np.float32)
    _check(load().xls_mlp_infer(m, px, X.shape[0], y.ctypes.data_as(c_void_p), 0))
    return y


def xls_mlp_loss_grad(m, X, y):
    X, px = _f32(X)
    y, py = _f32(y)
    loss = c_double()
    grad = np.zeros(N_MLP_PARAMS)
    _check(load().xls_mlp_loss_grad(m, px, py, X.shape[0], byref(loss), grad.ctypes.data_as(c_void_p), 0))
    return loss.value, grad


def xls_mlp_train_step(m, X, y, lr):
    X, px = _f32(X)
    y, py = _f32(y)
    loss = c_double()
    _check(load().xls_mlp_train_step(m, px, py, X.shape[0], float(lr), byref(loss), 0))
    return loss.value


def xls_descriptors(g, n_points):
    X = np.zeros((n_points, 32), dtype=np.float32)
    _check(load().xls_descriptors(g, X.ctypes.data_as(c_void_p), 0))
    return X


def xls_learned_start(g, m, n_electrons, n_points):
    rho = np.zeros(n_points)
    _check(load().xls_learned_start(g, m, float(n_electrons), rho.ctypes.data_as(c_void_p), 0))
    return rho


def xls_set_graphs(g, on):
    _check(load().xls_set_graphs(g, int(bool(on))))


def xls_scf_setup(g, n_electrons, kT, degree, n_passes=1, beta=0.3, kappa=0.5, history=7, pulay_period=2):
    _check(load().xls_scf_setup(g, float(n_electrons), float(kT), int(degree), int(n_passes), float(beta),
                                float(kappa), int(history), int(pulay_period)))


def xls_scf_step(g, rho):
    """One SCF step; rho (global grid, float64: a contiguous numpy array or a CUDA tensor) is
    replaced by the mixed next input density.  Returns (residual, energy, mu)."""
    res, en, mu = c_double(), c_double(), c_double()
    if hasattr(rho, "data_ptr"):
        _check(load().xls_scf_step(g, c_void_p(rho.data_ptr()), 1, byref(res), byref(en), byref(mu)))
    else:
        assert rho.dtype == np.float64 and rho.flags.c_contiguous
        _check(load().xls_scf_step(g, rho.ctypes.data_as(c_void_p), 0, byref(res), byref(en), byref(mu)))
    return res.value, en.value, mu.value


def xls_get_kernel_times(g):
    ms = np.zeros(8)
    cnt = np.zeros(8, dtype=np.int32)
    _check(load().xls_get_kernel_times(g, ms.ctypes.data_as(c_void_p), cnt.ctypes.data_as(c_void_p)))
    return ms, cnt


def xls_gram_noalloc(psi_f, hpsi_f, Ms_out, Hs_out, stream=None):
    """Allocation-free Gram of one block (see include/xls.h): psi_f, hpsi_f are contiguous CUDA
    float32 tensors of shape (n_states, n_points); Ms_out, Hs_out CUDA float64 (n_states, n_states)."""
    import torch
    for t in (psi_f, hpsi_f, Ms_out, Hs_out):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
            raise ValueError("xls_gram_noalloc takes contiguous CUDA tensors")
    if psi_f.dtype != torch.float32 or hpsi_f.dtype != torch.float32:
        raise TypeError("xls_gram_noalloc: psi_f and hpsi_f must be float32")
    if Ms_out.dtype != torch.float64 or Hs_out.dtype != torch.float64:
        raise TypeError("xls_gram_noalloc: Ms_out and Hs_out must be float64")
    if psi_f.dim() != 2 or tuple(hpsi_f.shape) != tuple(psi_f.shape):
        raise ValueError("xls_gram_noalloc: psi_f and hpsi_f must both be (n_states, n_points)")
    ns, nd = psi_f.shape
    if tuple(Ms_out.shape) != (ns, ns) or tuple(Hs_out.shape) != (ns, ns):
        raise ValueError(f"xls_gram_noalloc: Ms_out and Hs_out must be ({ns}, {ns})")
    dev = torch.cuda.current_device()
    if any(t.device.index != dev for t in (psi_f, hpsi_f, Ms_out, Hs_out)):
        raise ValueError("xls_gram_noalloc: every tensor must be on the current CUDA device")
    if stream is None:   # ordered after the torch work that produced the inputs
        stream = torch.cuda.current_stream().cuda_stream
    _check(load().xls_gram_noalloc(c_void_p(psi_f.data_ptr()), c_void_p(hpsi_f.data_ptr()), int(nd), int(ns),
                                   c_void_p(Ms_out.data_ptr()), c_void_p(Hs_out.data_ptr()),
                                   c_void_p(stream) if stream else None))
    return Ms_out, Hs_out


class Grid:
    """Owner of an xls_grid handle built from a synthetic workload description (any object
    with L, n, core_lo, core_n, buf, n_states, pos, species_index, species attributes)."""

    def __init__(self, w, precision=XLS_FP64, hbm_budget_bytes=0, stream=None):
        self.w = w
        self.precision = precision
        self.h = xls_grid_create(w.L, w.n, w.core_lo, w.core_n, w.buf, w.n_states, precision, hbm_budget_bytes, stream)

    def close(self):
        if self.h is not None:
            xls_grid_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_hamiltonian(self, veff):
        xls_hamiltonian_set(self.h, veff, self.w.pos, self.w.species_index, self.w.species)
