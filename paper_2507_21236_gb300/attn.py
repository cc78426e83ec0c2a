"""Thin ctypes binding of libattn (include/attn.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
computation of its own: arrays are passed as pointers (numpy for host
buffers; torch CUDA tensors or integer addresses for device buffers), handles
are opaque ``ctypes.c_void_p`` values, and a non-zero status raises
``AttnError`` with the library's message. The library has no CPU fallback:
if ``libattn.so`` is missing this module raises on import of the library.
"""
import ctypes
import os

import numpy as np

from . import _build

ATTN_F64, ATTN_F32, ATTN_TF32, ATTN_BF16 = 0, 1, 2, 3
STATUS = {0: "ATTN_OK", 1: "ATTN_EINVAL", 2: "ATTN_ENOMEM", 3: "ATTN_ECUDA", 4: "ATTN_ENONFINITE",
          5: "ATTN_ENOTISOMETRIC", 6: "ATTN_ENOTCONVERGED", 7: "ATTN_ETIMEOUT", 8: "ATTN_EUNSUPPORTED"}


class AttnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class attn_config(ctypes.Structure):
    _fields_ = [("lanczos_depth", ctypes.c_int), ("lanczos_tol", ctypes.c_double),
                ("de_max_iter", ctypes.c_int), ("de_rel_dev", ctypes.c_double),
                ("s_ttn", ctypes.c_int), ("matvec_dtype", ctypes.c_int),
                ("refine_steps", ctypes.c_int), ("refine_tol", ctypes.c_double),
                ("use_graphs", ctypes.c_int), ("refine_inner", ctypes.c_int),
                ("f64_split", ctypes.c_int), ("report_unconverged", ctypes.c_int),
                ("wait_limit_log2", ctypes.c_int), ("compress_terms", ctypes.c_int),
                ("de_method", ctypes.c_int), ("tc_schedule", ctypes.c_int),
                ("lanczos_basis", ctypes.c_int)]


class attn_heff_desc(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int * 3), ("h_int", ctypes.c_void_p * 3), ("n_pair", ctypes.c_int * 3),
                ("pair_a", ctypes.c_void_p * 3), ("pair_b", ctypes.c_void_p * 3),
                ("n_triple", ctypes.c_int), ("triple", ctypes.c_void_p * 3)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_PP = ctypes.POINTER(ctypes.c_void_p)
_PI = ctypes.POINTER(ctypes.c_int)
_PD = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "attn_config_default": [ctypes.POINTER(attn_config)],
    "attn_create": [ctypes.POINTER(attn_config), _P, _PP],
    "attn_destroy": [_P],
    "attn_set_config": [_P, ctypes.POINTER(attn_config)],
    "attn_get_config": [_P, ctypes.POINTER(attn_config)],
    "attn_sync": [_P],
    "attn_kernel_launches": [_P, ctypes.POINTER(ctypes.c_uint64)],
    "attn_profile_enable": [_P, _I],
    "attn_profile_read": [_P, _I, _PD, _PI, _PD],
    "attn_model_tfim": [_P, _I, _D, _PP],
    "attn_model_tri_heisenberg": [_P, _I, _D, _PP],
    "attn_model_terms": [_P, _I, _I, _PI, _PI, _PD, _PP],
    "attn_model_destroy": [_P],
    "attn_model_info": [_P, _PI, _PI],
    "attn_state_create": [_P, _P, _I, ctypes.POINTER(_PD), _PP],
    "attn_state_destroy": [_P],
    "attn_state_info": [_P, _PI, _PI, _PI],
    "attn_node_shape": [_P, _I, _PI],
    "attn_node_neighbour": [_P, _I, _I, _PI, _PI, _PI],
    "attn_node_get": [_P, _I, _PD],
    "attn_node_set": [_P, _I, _PD],
    "attn_node_device_ptr": [_P, _I, ctypes.POINTER(_P)],
    "attn_move_centre": [_P, _I],
    "attn_isometry_error": [_P, _PD],
    "attn_de_place": [_P, _I, _PI],
    "attn_de_sites": [_P, _PI],
    "attn_de_set": [_P, _I, _PD],
    "attn_de_get": [_P, _I, _PD],
    "attn_map_hamiltonian": [_P],
    "attn_hamiltonian_info": [_P, _PI, _PI],
    "attn_heff_counts": [_P, _I, _PI],
    "attn_heff_create": [_P, ctypes.POINTER(attn_heff_desc), _PP],
    "attn_heff_build": [_P, _I, _PP],
    "attn_heff_destroy": [_P],
    "attn_heff_info": [_P, _PI, _PI, _PD],
    "attn_heff_apply": [_P, _P, _P, _I],
    "attn_heff_apply_host": [_P, _PD, _PD, _I],
    "attn_eigsolve": [_P, _P, _PD, _PI],
    "attn_local_step": [_P, _I, _PD],
    "attn_ttn_sweep": [_P, _PD],
    "attn_energy": [_P, _PD],
    "attn_de_update": [_P, _PD],
    "attn_de_energies": [_P, _PD],
    "attn_sweep": [_P, _PD],
    "attn_mlp_param_count": [_PI],
    "attn_mlp_create": [_P, ctypes.POINTER(ctypes.c_float), _PP],
    "attn_mlp_destroy": [_P],
    "attn_mlp_get_params": [_P, ctypes.POINTER(ctypes.c_float)],
    "attn_mlp_predict": [_P, _I, _PD, _PD],
    "attn_mlp_loss_grad": [_P, _I, _PD, _PD, _PD, ctypes.POINTER(ctypes.c_float)],
    "attn_mlp_train": [_P, _I, _PD, _PD, _I, _D, _PD],
    "attn_set_learned_init": [_P, _P],
    "attn_de_training_pairs": [_P, _PD, _PD],
    "attn_learned_init_report": [_P, _PI, _PI],
    "attn_heff_apply_f64_static": [ctypes.POINTER(attn_heff_desc), _P, _P, _P],
    "attn_set_allocator": [_P, _P, _P],
    "attn_renormalise": [_P, _I, _I, _PI],
    "attn_link_operators": [_P, _I, _I, _PI, _PI, _PI, _PD],
    "attn_state_save": [_P, ctypes.c_char_p],
    "attn_state_load": [_P, ctypes.c_char_p],
    "attn_eigsolve_host": [_P, _PD, _PD, _PI],
    "attn_de_update_one": [_P, _I, _PD],
    "attn_de_environment": [_P, _I, _PD, _PD, _PD],
    "attn_rdm2": [_P, _I, _PD],
    "attn_measure": [_P, _I, _PI, _PI, _PD, _PD],
    "attn_correlation_matrix": [_P, _PD, _PD, _PD],
}

# C callback types of attn_set_allocator
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p)
_allocator_refs = []  # callbacks stay referenced while the library may call them

_lib = None


def library_path():
    return _build.LIB


def load(path=None):
    """Load libattn.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with `python -m paper_2507_21236_gb300._build` "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.attn_last_error.restype = ctypes.c_char_p
    lib.attn_last_error.argtypes = []
    lib.attn_version.restype = ctypes.c_char_p
    lib.attn_version.argtypes = []
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS) + ["attn_last_error", "attn_version"]


def _check(st):
    if st != 0:
        raise AttnError(st, load().attn_last_error().decode())


def _ptr(a):
    """Device address of a torch tensor / int, or None."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    return a.data_ptr()


def _host_d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_PD)


# --------------------------------------------------------------------- context
def attn_last_error():
    return load().attn_last_error().decode()


def attn_version():
    return load().attn_version().decode()


def attn_config_default():
    cfg = attn_config()
    _check(load().attn_config_default(ctypes.byref(cfg)))
    return cfg


def attn_create(cfg=None, stream=None):
    """Create a context; ``stream`` is a cudaStream_t as int (e.g. torch's cuda_stream)."""
    h = ctypes.c_void_p()
    _check(load().attn_create(ctypes.byref(cfg) if cfg is not None else None, stream, ctypes.byref(h)))
    return h


def attn_destroy(ctx):
    _check(load().attn_destroy(ctx))


def attn_set_config(ctx, cfg):
    _check(load().attn_set_config(ctx, ctypes.byref(cfg)))


def attn_get_config(ctx):
    cfg = attn_config()
    _check(load().attn_get_config(ctx, ctypes.byref(cfg)))
    return cfg


def attn_sync(ctx):
    _check(load().attn_sync(ctx))


def attn_kernel_launches(ctx):
    c = ctypes.c_uint64()
    _check(load().attn_kernel_launches(ctx, ctypes.byref(c)))
    return c.value


def attn_profile_enable(ctx, enable=True):
    _check(load().attn_profile_enable(ctx, 1 if enable else 0))


def attn_profile_read(ctx, kernel_id):
    """(total device ms, launches, algorithmic FLOPs) of the recorded launches."""
    ms, n, fl = ctypes.c_double(), ctypes.c_int(), ctypes.c_double()
    _check(load().attn_profile_read(ctx, kernel_id, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(fl)))
    return ms.value, n.value, fl.value


# ---------------------------------------------------------------------- models
def attn_model_tfim(ctx, L, h):
    m = ctypes.c_void_p()
    _check(load().attn_model_tfim(ctx, L, h, ctypes.byref(m)))
    return m


def attn_model_tri_heisenberg(ctx, L, J=1.0):
    m = ctypes.c_void_p()
    _check(load().attn_model_tri_heisenberg(ctx, L, J, ctypes.byref(m)))
    return m


def attn_model_terms(ctx, n_sites, terms):
    """``terms``: list of (ascending sites tuple, real 2^k x 2^k operator)."""
    n = len(terms)
    ns = np.zeros(n, dtype=np.int32)
    sites = np.zeros(3 * n, dtype=np.int32)
    ops = np.zeros(64 * n, dtype=np.float64)
    for t, (s, op) in enumerate(terms):
        ns[t] = len(s)
        sites[3 * t:3 * t + len(s)] = s
        op = np.asarray(op, dtype=np.float64).reshape(-1)
        ops[64 * t:64 * t + op.size] = op
    m = ctypes.c_void_p()
    _check(load().attn_model_terms(ctx, n_sites, n, ns.ctypes.data_as(_PI), sites.ctypes.data_as(_PI),
                                   ops.ctypes.data_as(_PD), ctypes.byref(m)))
    return m


def attn_model_destroy(model):
    _check(load().attn_model_destroy(model))


def attn_model_info(model):
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(load().attn_model_info(model, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


# ----------------------------------------------------------------------- state
def attn_state_create(ctx, model, m, raw_tensors):
    arrs = [np.ascontiguousarray(t, dtype=np.float64) for t in raw_tensors]
    ptrs = (_PD * len(arrs))(*[a.ctypes.data_as(_PD) for a in arrs])
    st = ctypes.c_void_p()
    _check(load().attn_state_create(ctx, model, m, ptrs, ctypes.byref(st)))
    return st


def attn_state_destroy(st):
    _check(load().attn_state_destroy(st))


def attn_state_info(st):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().attn_state_info(st, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def attn_node_shape(st, node):
    s = (ctypes.c_int * 3)()
    _check(load().attn_node_shape(st, node, s))
    return tuple(s)


def attn_node_neighbour(st, node, slot):
    k, i, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().attn_node_neighbour(st, node, slot, ctypes.byref(k), ctypes.byref(i), ctypes.byref(b)))
    return k.value, i.value, b.value


def attn_node_get(st, node):
    out = np.empty(attn_node_shape(st, node), dtype=np.float64)
    _check(load().attn_node_get(st, node, out.ctypes.data_as(_PD)))
    return out


def attn_node_set(st, node, t):
    a, p = _host_d(t)
    _check(load().attn_node_set(st, node, p))


def attn_node_device_ptr(st, node):
    p = ctypes.c_void_p()
    _check(load().attn_node_device_ptr(st, node, ctypes.byref(p)))
    return p.value


def attn_move_centre(st, node):
    _check(load().attn_move_centre(st, node))


def attn_isometry_error(st):
    e = ctypes.c_double()
    _check(load().attn_isometry_error(st, ctypes.byref(e)))
    return e.value


# --------------------------------------------------------------- disentanglers
def attn_de_place(st, max_de):
    n = ctypes.c_int()
    _check(load().attn_de_place(st, max_de, ctypes.byref(n)))
    return n.value


def attn_de_sites(st, n):
    out = np.zeros(2 * max(n, 1), dtype=np.int32)
    _check(load().attn_de_sites(st, out.ctypes.data_as(_PI)))
    return [tuple(int(v) for v in out[2 * k:2 * k + 2]) for k in range(n)]


def attn_de_set(st, k, u):
    a, p = _host_d(np.asarray(u).reshape(16))
    _check(load().attn_de_set(st, k, p))


def attn_de_get(st, k):
    out = np.zeros(16)
    _check(load().attn_de_get(st, k, out.ctypes.data_as(_PD)))
    return out.reshape(4, 4)


def attn_map_hamiltonian(st):
    _check(load().attn_map_hamiltonian(st))


def attn_hamiltonian_info(st):
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(load().attn_hamiltonian_info(st, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def attn_heff_counts(st, node):
    c = (ctypes.c_int * 5)()
    _check(load().attn_heff_counts(st, node, c))
    return tuple(c)


# ----------------------------------------------------------------------- H_eff
def attn_heff_create(ctx, m, h_int=(None, None, None), pairs=None, triples=None):
    """Explicit H_eff from DEVICE operator stacks (torch CUDA float64 tensors).

    ``pairs``: dict kind -> (A stack, B stack) with kind 0 = slots (0,1),
    1 = (0,2), 2 = (1,2); ``triples``: (O0, O1, O2) stacks or None."""
    d = attn_heff_desc()
    for s in range(3):
        d.m[s] = m[s]
        d.h_int[s] = _ptr(h_int[s])
    for k, (a, b) in (pairs or {}).items():
        d.n_pair[k] = a.shape[0]
        d.pair_a[k] = _ptr(a)
        d.pair_b[k] = _ptr(b)
    if triples is not None:
        d.n_triple = triples[0].shape[0]
        for s in range(3):
            d.triple[s] = _ptr(triples[s])
    h = ctypes.c_void_p()
    _check(load().attn_heff_create(ctx, ctypes.byref(d), ctypes.byref(h)))
    return h


def _desc(m, h_int=(None, None, None), pairs=None, triples=None):
    d = attn_heff_desc()
    for s in range(3):
        d.m[s] = m[s]
        d.h_int[s] = _ptr(h_int[s])
    for k, (a, b) in (pairs or {}).items():
        d.n_pair[k] = a.shape[0]
        d.pair_a[k] = _ptr(a)
        d.pair_b[k] = _ptr(b)
    if triples is not None:
        d.n_triple = triples[0].shape[0]
        for s in range(3):
            d.triple[s] = _ptr(triples[s])
    return d


def attn_heff_apply_f64_static(m, x_dev, y_dev, h_int=(None, None, None), pairs=None, triples=None, stream=None):
    """Allocation-free FP64 H_eff apply straight from device operator arrays."""
    d = _desc(m, h_int, pairs, triples)
    _check(load().attn_heff_apply_f64_static(ctypes.byref(d), _ptr(x_dev), _ptr(y_dev), stream))


def attn_heff_build(st, node):
    h = ctypes.c_void_p()
    _check(load().attn_heff_build(st, node, ctypes.byref(h)))
    return h


def attn_heff_destroy(h):
    _check(load().attn_heff_destroy(h))


def attn_heff_info(h):
    npair = (ctypes.c_int * 3)()
    nt = ctypes.c_int()
    fl = ctypes.c_double()
    _check(load().attn_heff_info(h, npair, ctypes.byref(nt), ctypes.byref(fl)))
    return tuple(npair), nt.value, fl.value


def attn_heff_apply(h, x_dev, y_dev, dtype=ATTN_F64):
    _check(load().attn_heff_apply(h, _ptr(x_dev), _ptr(y_dev), dtype))


def attn_heff_apply_host(h, x, dtype=ATTN_F64):
    xa, xp = _host_d(x)
    y = np.empty_like(xa)
    _check(load().attn_heff_apply_host(h, xp, y.ctypes.data_as(_PD), dtype))
    return y


def attn_eigsolve(h, T_dev):
    th = ctypes.c_double()
    it = ctypes.c_int()
    _check(load().attn_eigsolve(h, _ptr(T_dev), ctypes.byref(th), ctypes.byref(it)))
    return th.value, it.value


# ---------------------------------------------------------------------- sweeps
def attn_local_step(st, node):
    e = ctypes.c_double()
    _check(load().attn_local_step(st, node, ctypes.byref(e)))
    return e.value


def attn_ttn_sweep(st):
    e = ctypes.c_double()
    _check(load().attn_ttn_sweep(st, ctypes.byref(e)))
    return e.value


def attn_energy(st):
    e = ctypes.c_double()
    _check(load().attn_energy(st, ctypes.byref(e)))
    return e.value


# ------------------------------------------------------------ disentangler update
def attn_de_update(st):
    d = ctypes.c_double()
    _check(load().attn_de_update(st, ctypes.byref(d)))
    return d.value


def attn_de_energies(st, n_de):
    out = np.zeros(2 * max(n_de, 1))
    _check(load().attn_de_energies(st, out.ctypes.data_as(_PD)))
    return out[:2 * n_de].reshape(n_de, 2)


def attn_sweep(st):
    e = ctypes.c_double()
    _check(load().attn_sweep(st, ctypes.byref(e)))
    return e.value


# ------------------------------------------------------- learned initialiser
_PF = ctypes.POINTER(ctypes.c_float)


def attn_mlp_param_count():
    n = ctypes.c_int()
    _check(load().attn_mlp_param_count(ctypes.byref(n)))
    return n.value


def attn_mlp_create(ctx, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    m = ctypes.c_void_p()
    _check(load().attn_mlp_create(ctx, p.ctypes.data_as(_PF), ctypes.byref(m)))
    return m


def attn_mlp_destroy(m):
    _check(load().attn_mlp_destroy(m))


def attn_mlp_get_params(m):
    out = np.empty(attn_mlp_param_count(), dtype=np.float32)
    _check(load().attn_mlp_get_params(m, out.ctypes.data_as(_PF)))
    return out


def attn_mlp_predict(m, rho):
    r, rp = _host_d(np.asarray(rho).reshape(-1, 16))
    u = np.empty_like(r)
    _check(load().attn_mlp_predict(m, r.shape[0], rp, u.ctypes.data_as(_PD)))
    return u.reshape(-1, 4, 4)


def attn_mlp_loss_grad(m, rho, ut):
    r, rp = _host_d(np.asarray(rho).reshape(-1, 16))
    t, tp = _host_d(np.asarray(ut).reshape(-1, 16))
    loss = ctypes.c_double()
    g = np.empty(attn_mlp_param_count(), dtype=np.float32)
    _check(load().attn_mlp_loss_grad(m, r.shape[0], rp, tp, ctypes.byref(loss), g.ctypes.data_as(_PF)))
    return loss.value, g


def attn_mlp_train(m, rho, ut, steps, lr):
    r, rp = _host_d(np.asarray(rho).reshape(-1, 16))
    t, tp = _host_d(np.asarray(ut).reshape(-1, 16))
    loss = ctypes.c_double()
    _check(load().attn_mlp_train(m, r.shape[0], rp, tp, steps, lr, ctypes.byref(loss)))
    return loss.value


def attn_set_learned_init(st, m):
    _check(load().attn_set_learned_init(st, m))


def attn_de_training_pairs(st, n_de):
    rho = np.zeros(16 * max(n_de, 1))
    u = np.zeros(16 * max(n_de, 1))
    _check(load().attn_de_training_pairs(st, rho.ctypes.data_as(_PD), u.ctypes.data_as(_PD)))
    return rho[:16 * n_de].reshape(n_de, 16), u[:16 * n_de].reshape(n_de, 4, 4)


def attn_learned_init_report(st):
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(load().attn_learned_init_report(st, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


# ----------------------------------------------------------- boundary additions
def attn_set_allocator(alloc=None, free=None):
    """Install Python callables alloc(bytes, device) -> address and free(address, bytes,
    device) as the library's device allocator (None, None: back to cudaMalloc)."""
    if alloc is None:
        _check(load().attn_set_allocator(None, None, None))
        return
    a = ALLOC_FN(lambda n, dev, user: alloc(n, dev))
    f = FREE_FN(lambda p, n, dev, user: free(p, n, dev))
    _allocator_refs.append((a, f))
    _check(load().attn_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None))


def attn_renormalise(st, node, slot):
    n = ctypes.c_int()
    _check(load().attn_renormalise(st, node, slot, ctypes.byref(n)))
    return n.value


def attn_link_operators(st, node, slot):
    """(dim, n_open, has_internal, internal operator [dim, dim])."""
    d, n, h = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().attn_link_operators(st, node, slot, ctypes.byref(d), None, None, None))
    out = np.zeros((d.value, d.value))
    _check(load().attn_link_operators(st, node, slot, ctypes.byref(d), ctypes.byref(n), ctypes.byref(h),
                                      out.ctypes.data_as(_PD)))
    return d.value, n.value, bool(h.value), out


def attn_state_save(st, path):
    _check(load().attn_state_save(st, os.fsencode(path)))


def attn_state_load(st, path):
    _check(load().attn_state_load(st, os.fsencode(path)))


def attn_eigsolve_host(h, T_host):
    """Eigensolve on a host float64 C-contiguous array, updated in place with the Ritz vector."""
    assert T_host.dtype == np.float64 and T_host.flags.c_contiguous
    th, it = ctypes.c_double(), ctypes.c_int()
    _check(load().attn_eigsolve_host(h, T_host.ctypes.data_as(_PD), ctypes.byref(th), ctypes.byref(it)))
    return th.value, it.value


def attn_de_update_one(st, k):
    d = ctypes.c_double()
    _check(load().attn_de_update_one(st, k, ctypes.byref(d)))
    return d.value


def attn_de_environment(st, k, u):
    ua, up = _host_d(np.asarray(u).reshape(16))
    g = np.zeros(16)
    e = ctypes.c_double()
    _check(load().attn_de_environment(st, k, up, g.ctypes.data_as(_PD), ctypes.byref(e)))
    return g.reshape(4, 4), e.value


def attn_rdm2(st, k):
    r = np.zeros(16)
    _check(load().attn_rdm2(st, k, r.ctypes.data_as(_PD)))
    return r.reshape(4, 4)


def attn_measure(st, observables):
    """``observables``: list of (sites, [2x2 operators]) with 1..4 distinct sites each."""
    n = len(observables)
    ns = np.zeros(max(n, 1), dtype=np.int32)
    sites = np.zeros(4 * max(n, 1), dtype=np.int32)
    ops = np.zeros(16 * max(n, 1))
    for q, (s, o) in enumerate(observables):
        ns[q] = len(s)
        sites[4 * q:4 * q + len(s)] = s
        for a, m in enumerate(o):
            ops[16 * q + 4 * a:16 * q + 4 * a + 4] = np.asarray(m, dtype=np.float64).reshape(4)
    out = np.zeros(max(n, 1))
    _check(load().attn_measure(st, n, ns.ctypes.data_as(_PI), sites.ctypes.data_as(_PI), ops.ctypes.data_as(_PD),
                               out.ctypes.data_as(_PD)))
    return out[:n]


def attn_correlation_matrix(st, oa, ob, n_sites):
    a, ap = _host_d(np.asarray(oa).reshape(4))
    b, bp = _host_d(np.asarray(ob).reshape(4))
    C = np.zeros((n_sites, n_sites))
    _check(load().attn_correlation_matrix(st, ap, bp, C.ctypes.data_as(_PD)))
    return C
