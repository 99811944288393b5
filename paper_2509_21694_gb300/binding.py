"""Thin ctypes binding of the C ABI declared in include/mpip.h.

Functions keep the C names (mp_create, mp_build_neighbors, mp_partition,
mp_energy_forces, mp_md_step, ...) and only marshal arguments: torch CUDA
tensors are passed as raw device pointers, the context runs on the caller's
current torch CUDA stream.  Every step of the computation runs in the
library's CUDA kernels; if libmpip.so is missing this module raises at
import time instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpip.so")

MP_OK = 0
MP_ERR_ARG, MP_ERR_TIMEOUT = -1, -9
MP_FP32, MP_BF16 = 0, 1
MP_HALO_GEOM, MP_HALO_BFS = 0, 1
MP_NVE, MP_LANGEVIN = 0, 1
ERRORS = {-1: "MP_ERR_ARG", -2: "MP_ERR_BOX_TOO_SMALL", -3: "MP_ERR_OVERLAP",
          -4: "MP_ERR_CAPACITY", -5: "MP_ERR_CUDA", -6: "MP_ERR_NOT_FINITE",
          -7: "MP_ERR_NOMEM", -8: "MP_ERR_UNSUPPORTED", -9: "MP_ERR_TIMEOUT",
          -10: "MP_ERR_TOO_LARGE"}


class MPError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__("%s failed: %s (%s)" % (what, ERRORS.get(code, code), _strerror(code)))


class mp_model_desc(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int32), ("F", ctypes.c_int32), ("lmax", ctypes.c_int32),
                ("n_layers_full", ctypes.c_int32), ("H", ctypes.c_int32),
                ("n_basis", ctypes.c_int32), ("p_env", ctypes.c_int32),
                ("head_hidden", ctypes.c_int32), ("r_cut", ctypes.c_double),
                ("n_avg", ctypes.c_double), ("rep_eps", ctypes.c_double),
                ("rep_sigma", ctypes.c_double)]


class mp_md_opts(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("n_parts", ctypes.c_int32), ("k_hops", ctypes.c_int32),
                ("halo_mode", ctypes.c_int32), ("use_head", ctypes.c_int32),
                ("forces_valid", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("thermostat", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("temperature", ctypes.c_double), ("friction", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("step0", ctypes.c_int64),
                ("d_part", ctypes.c_void_p), ("skin", ctypes.c_double),
                ("h_builds", ctypes.POINTER(ctypes.c_int64))]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libmpip.so is not built (run paper_2509_21694_gb300/build.py)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "mp_weights_count": (I32, [ctypes.POINTER(mp_model_desc), ctypes.POINTER(I64)]),
        "mp_create": (I32, [PP, ctypes.POINTER(mp_model_desc), P, I64, P]),
        "mp_set_stream": (I32, [P, P]),
        "mp_set_head": (I32, [P, P, I64]),
        "mp_destroy": (None, [P]),
        "mp_build_neighbors": (I32, [P, P, I64, ctypes.POINTER(D), PP]),
        "mp_graph_info": (I32, [P, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "mp_graph_export": (I32, [P, P, P, P]),
        "mp_graph_free": (None, [P]),
        "mp_partition": (I32, [P, P, I32, I32, I32, PP, ctypes.POINTER(D)]),
        "mp_partition_assign": (I32, [P, P, P, I32, I32, PP, ctypes.POINTER(D)]),
        "mp_graph_partition": (I32, [P, P, I32, D, ctypes.c_uint64, P, ctypes.POINTER(I64)]),
        "mp_partition_host_bisect": (I32, [I32, P, P, P, P, I32, ctypes.c_uint64, P]),
        "mp_plan_info": (I32, [P, I32, ctypes.POINTER(I64), ctypes.POINTER(I64),
                               ctypes.POINTER(I64)]),
        "mp_plan_export": (I32, [P, I32, P, P]),
        "mp_plan_free": (None, [P]),
        "mp_energy_forces": (I32, [P, P, P, P, P, I32, I32, I32, P, P, P]),
        "mp_energy_forces_stress": (I32, [P, P, P, P, P, I32, I32, I32, P, P, P, P]),
        "mp_energy_forces_parts": (I32, [P, P, P, P, P, I32, I32, I32, I32, I32, P, P, P]),
        "mp_verlet_first_half": (I32, [P, P, P, P, P, I64, ctypes.POINTER(D), D]),
        "mp_verlet_second_half": (I32, [P, P, P, P, I64, D, P]),
        "mp_layer_stats": (I32, [P, P, P, P, I32, I32, P, P]),
        "mp_md_step": (I32, [P, P, P, P, P, P, I64, ctypes.POINTER(D), D, I32,
                             ctypes.POINTER(mp_md_opts), P]),
        "mp_kernel_launches": (I32, [ctypes.POINTER(I64)]),
        "mp_timing_enable": (I32, [P, I32]),
        "mp_timing_read": (I32, [P, P, P, P, P]),
        "mp_energy_sum_noalloc": (I32, [P, I64, P, P]),
        "mp_wait_selftest": (I32, [P, I64, I32]),
        "mp_head_count": (I32, [P, ctypes.POINTER(I64)]),
        "mp_head_loss_grad": (I32, [P, P, P, P, I32, I32, P, P, D, P, P]),
        "mp_head_adam_step": (I32, [P, P, D, D, D, D, I64]),
        "mp_head_get": (I32, [P, P, I64]),
        "mp_strerror": (ctypes.c_char_p, [I32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def _strerror(code: int) -> str:
    return _lib.mp_strerror(code).decode()


def _check(rc: int, what: str):
    if rc != MP_OK:
        raise MPError(rc, what)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


# ---------------------------------------------------------------- weights --

def desc_struct(desc) -> mp_model_desc:
    return mp_model_desc(desc.n_species, desc.F, desc.lmax, desc.n_layers_full, desc.H,
                         desc.n_basis, desc.p_env, desc.head_hidden, desc.r_cut, desc.n_avg,
                         desc.rep_eps, desc.rep_sigma)


def head_vector(w: dict) -> np.ndarray:
    return np.concatenate([np.ravel(w[k]) for k in ("head_W1", "head_b1", "head_W2", "head_b2")])


def pack_weights(w: dict, desc) -> np.ndarray:
    """Flat float64 vector in the order mp_create documents."""
    parts = [w["emb"], w["e0"], w["w_out"], head_vector(w)]
    for t in range(desc.n_layers_full):
        parts += [w["W1"][t], w["W2"][t], w["W3"][t], w["W0"][t], w["U1"][t]]
        if desc.lmax >= 2:
            parts.append(w["U2"][t])
        parts += [w["b"][t], w["V1"][t]]
        if desc.lmax >= 2:
            parts.append(w["V2"][t])
    out = np.ascontiguousarray(np.concatenate([np.ravel(np.asarray(p, np.float64)) for p in parts]))
    n = ctypes.c_int64()
    _check(_lib.mp_weights_count(ctypes.byref(desc_struct(desc)), ctypes.byref(n)), "mp_weights_count")
    if out.size != n.value:
        raise ValueError("weight vector has %d entries, expected %d" % (out.size, n.value))
    return out


# --------------------------------------------------------- C-named calls --

def mp_create(desc, weights: dict, stream: int | None = None) -> int:
    vec = pack_weights(weights, desc)
    h = ctypes.c_void_p()
    ds = desc_struct(desc)
    _check(_lib.mp_create(ctypes.byref(h), ctypes.byref(ds), vec.ctypes.data, vec.size,
                          _stream() if stream is None else stream), "mp_create")
    return h.value


def mp_destroy(ctx: int):
    _lib.mp_destroy(ctx)


def mp_set_stream(ctx: int, stream: int):
    _check(_lib.mp_set_stream(ctx, stream), "mp_set_stream")


def mp_set_head(ctx: int, head: np.ndarray):
    head = np.ascontiguousarray(head, dtype=np.float64)
    _check(_lib.mp_set_head(ctx, head.ctypes.data, head.size), "mp_set_head")


def mp_build_neighbors(ctx: int, pos: torch.Tensor, box) -> int:
    b = (ctypes.c_double * 3)(*[float(v) for v in box])
    g = ctypes.c_void_p()
    _check(_lib.mp_build_neighbors(ctx, _ptr(pos), pos.shape[0], b, ctypes.byref(g)),
           "mp_build_neighbors")
    return g.value


def mp_graph_info(g: int):
    n, e = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.mp_graph_info(g, ctypes.byref(n), ctypes.byref(e)), "mp_graph_info")
    return n.value, e.value


def mp_graph_export(g: int):
    n, ne = mp_graph_info(g)
    dev = torch.device("cuda")
    recv = torch.empty(ne, dtype=torch.int32, device=dev)
    send = torch.empty(ne, dtype=torch.int32, device=dev)
    shift = torch.empty(ne, dtype=torch.int8, device=dev)
    if ne:
        _check(_lib.mp_graph_export(g, _ptr(recv), _ptr(send), _ptr(shift)), "mp_graph_export")
    return recv, send, shift


def mp_graph_free(g: int):
    _lib.mp_graph_free(g)


def mp_partition(ctx: int, g: int, n_parts: int, k_hops: int, mode: int = MP_HALO_GEOM):
    p = ctypes.c_void_p()
    H = ctypes.c_double()
    _check(_lib.mp_partition(ctx, g, n_parts, k_hops, mode, ctypes.byref(p), ctypes.byref(H)),
           "mp_partition")
    return p.value, H.value


def mp_partition_assign(ctx: int, g: int, part: torch.Tensor, n_parts: int, k_hops: int):
    """Plan with the roots of ``part`` (int32 [n] device, caller order) and BFS halos."""
    assert part.dtype == torch.int32 and part.is_cuda and part.is_contiguous()
    p = ctypes.c_void_p()
    H = ctypes.c_double()
    _check(_lib.mp_partition_assign(ctx, g, _ptr(part), n_parts, k_hops, ctypes.byref(p),
                                    ctypes.byref(H)), "mp_partition_assign")
    return p.value, H.value


def mp_graph_partition(ctx: int, g: int, n_parts: int, imbalance: float = 0.03, seed: int = 0,
                       part: torch.Tensor | None = None):
    """(part int32 [n] device in caller order, number of cut edges)."""
    n, _ = mp_graph_info(g)
    if part is None:
        part = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    cut = ctypes.c_int64()
    _check(_lib.mp_graph_partition(ctx, g, n_parts, imbalance, seed, _ptr(part),
                                   ctypes.byref(cut)), "mp_graph_partition")
    return part[:n], cut.value


def mp_partition_host_bisect(row_ptr, col, n_parts: int, seed: int = 0, edge_w=None,
                             vertex_w=None) -> np.ndarray:
    """Recursive greedy bisection of a host CSR graph (numpy arrays); host only."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = len(row_ptr) - 1
    ew = None if edge_w is None else np.ascontiguousarray(edge_w, dtype=np.int32)
    vw = None if vertex_w is None else np.ascontiguousarray(vertex_w, dtype=np.int32)
    m = int(row_ptr[-1]) if n >= 0 and len(row_ptr) else -1
    if n < 0 or len(col) != m or (ew is not None and len(ew) != m) or (vw is not None and len(vw) != n):
        raise ValueError("row_ptr, col and the weights do not describe one CSR graph")
    part = np.zeros(max(n, 1), dtype=np.int32)
    _check(_lib.mp_partition_host_bisect(n, row_ptr.ctypes.data, col.ctypes.data if len(col) else None,
                                         None if ew is None else ew.ctypes.data,
                                         None if vw is None else vw.ctypes.data, n_parts, seed,
                                         part.ctypes.data), "mp_partition_host_bisect")
    return part[:n]


def mp_plan_info(plan: int, p: int):
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.mp_plan_info(plan, p, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "mp_plan_info")
    return a.value, b.value, c.value


def mp_plan_export(plan: int, p: int):
    n_ext, _, _ = mp_plan_info(plan, p)
    gid = torch.empty(max(n_ext, 1), dtype=torch.int32, device="cuda")
    root = torch.empty(max(n_ext, 1), dtype=torch.uint8, device="cuda")
    _check(_lib.mp_plan_export(plan, p, _ptr(gid), _ptr(root)), "mp_plan_export")
    return gid[:n_ext], root[:n_ext]


def mp_plan_free(plan: int):
    _lib.mp_plan_free(plan)


def mp_energy_forces(ctx: int, pos: torch.Tensor, species: torch.Tensor, g: int, plan,
                     n_layers: int, precision: int = MP_FP32, use_head: bool = False,
                     energy: torch.Tensor | None = None, forces: torch.Tensor | None = None,
                     e_atom: torch.Tensor | None = None):
    n = pos.shape[0]
    if energy is None:
        energy = torch.empty(1, dtype=torch.float64, device=pos.device)
    if forces is None:
        forces = torch.empty(n, 3, dtype=torch.float32, device=pos.device)
    _check(_lib.mp_energy_forces(ctx, _ptr(pos), _ptr(species), g, plan or None, n_layers,
                                 precision, int(use_head), _ptr(energy), _ptr(forces),
                                 _ptr(e_atom)), "mp_energy_forces")
    return energy, forces, e_atom


def mp_energy_forces_stress(ctx: int, pos: torch.Tensor, species: torch.Tensor, g: int, plan,
                            n_layers: int, precision: int = MP_FP32, use_head: bool = False,
                            e_atom: torch.Tensor | None = None):
    """(E, F, e_atom, stress[3, 3]) with stress = (1/V) dE/d(strain) in eV/A^3."""
    n = pos.shape[0]
    energy = torch.empty(1, dtype=torch.float64, device=pos.device)
    forces = torch.empty(n, 3, dtype=torch.float32, device=pos.device)
    stress = torch.empty(3, 3, dtype=torch.float64, device=pos.device)
    _check(_lib.mp_energy_forces_stress(ctx, _ptr(pos), _ptr(species), g, plan or None, n_layers,
                                        precision, int(use_head), _ptr(energy), _ptr(forces),
                                        _ptr(e_atom), _ptr(stress)), "mp_energy_forces_stress")
    return energy, forces, e_atom, stress


def mp_energy_forces_parts(ctx: int, pos: torch.Tensor, species: torch.Tensor, g: int,
                           plan: int, part_begin: int, part_end: int, n_layers: int,
                           precision: int = MP_FP32, use_head: bool = False,
                           energy: torch.Tensor | None = None,
                           forces64: torch.Tensor | None = None,
                           e_atom: torch.Tensor | None = None):
    """FP64 shares (energy [1], forces [n, 3]) of partitions part_begin ..
    part_end - 1 of ``plan``."""
    n = pos.shape[0]
    if energy is None:
        energy = torch.empty(1, dtype=torch.float64, device=pos.device)
    if forces64 is None:
        forces64 = torch.empty(n, 3, dtype=torch.float64, device=pos.device)
    assert energy.dtype == torch.float64 and forces64.dtype == torch.float64
    assert forces64.numel() == 3 * n
    _check(_lib.mp_energy_forces_parts(ctx, _ptr(pos), _ptr(species), g, plan, part_begin,
                                       part_end, n_layers, precision, int(use_head),
                                       _ptr(energy), _ptr(forces64), _ptr(e_atom)),
           "mp_energy_forces_parts")
    return energy, forces64, e_atom


def mp_verlet_first_half(ctx: int, pos, vel, forces64, mass, box, dt: float):
    b = (ctypes.c_double * 3)(*[float(v) for v in box])
    _check(_lib.mp_verlet_first_half(ctx, _ptr(pos), _ptr(vel), _ptr(forces64), _ptr(mass),
                                     pos.shape[0], b, dt), "mp_verlet_first_half")


def mp_verlet_second_half(ctx: int, vel, forces64, mass, dt: float, ke: torch.Tensor):
    assert ke.dtype == torch.float64 and ke.numel() >= 1
    _check(_lib.mp_verlet_second_half(ctx, _ptr(vel), _ptr(forces64), _ptr(mass), vel.shape[0],
                                      dt, _ptr(ke)), "mp_verlet_second_half")


def mp_layer_stats(ctx: int, pos: torch.Tensor, species: torch.Tensor, g: int, n_layers: int,
                   precision: int = MP_FP32):
    """(MFS, CKA) numpy arrays of length n_layers for the transitions t -> t + 1."""
    mfs = np.zeros(n_layers, dtype=np.float64)
    cka = np.zeros(n_layers, dtype=np.float64)
    _check(_lib.mp_layer_stats(ctx, _ptr(pos), _ptr(species), g, n_layers, precision,
                               mfs.ctypes.data, cka.ctypes.data), "mp_layer_stats")
    return mfs, cka


def mp_md_step(ctx: int, pos, vel, forces, mass, species, box, dt: float, n_steps: int,
               n_layers: int, precision: int = MP_FP32, n_parts: int = 1, k_hops: int = 0,
               halo_mode: int = MP_HALO_GEOM, use_head: bool = False, forces_valid: bool = False,
               check_every: int = 0, ledger: bool = True, thermostat: int = MP_NVE,
               temperature: float = 0.0, friction: float = 0.0, seed: int = 0, step0: int = 0,
               part: torch.Tensor | None = None, skin: float = 0.0, builds: list | None = None):
    """``part``: per-atom roots (int32 [n] device, caller order) instead of z slabs.
    ``skin`` (A): Verlet-skin reuse of neighbours and partitions; ``builds``, a
    list, receives the number of list builds done by the call."""
    if part is not None:
        assert part.dtype == torch.int32 and part.is_cuda and part.is_contiguous()
    nb = ctypes.c_int64(0)
    opts = mp_md_opts(n_layers, precision, n_parts, k_hops, halo_mode, int(use_head),
                      int(forces_valid), check_every, thermostat, 0, temperature, friction,
                      seed, step0, _ptr(part) if part is not None else None, float(skin),
                      ctypes.pointer(nb))
    b = (ctypes.c_double * 3)(*[float(v) for v in box])
    led = np.zeros((max(n_steps, 1), 3), dtype=np.float64)
    _check(_lib.mp_md_step(ctx, _ptr(pos), _ptr(vel), _ptr(forces), _ptr(mass), _ptr(species),
                           pos.shape[0], b, dt, n_steps, ctypes.byref(opts),
                           led.ctypes.data if ledger else None), "mp_md_step")
    if builds is not None:
        builds.append(nb.value)
    return led[:n_steps]


TIMERS = ("neighbors", "partition", "edge_fwd", "edge_bwd", "node_fwd", "node_bwd",
          "edge_fwd_l0", "edge_bwd_l0", "node_fwd_l0", "node_bwd_l0")


def mp_timing_enable(ctx: int, enable: bool = True):
    _check(_lib.mp_timing_enable(ctx, int(enable)), "mp_timing_enable")


def mp_timing_read(ctx: int) -> dict:
    n = len(TIMERS)
    ms = np.zeros(n, np.float64)
    la, ed, at = (np.zeros(n, np.int64) for _ in range(3))
    _check(_lib.mp_timing_read(ctx, ms.ctypes.data, la.ctypes.data, ed.ctypes.data,
                               at.ctypes.data), "mp_timing_read")
    return {name: {"ms": float(ms[q]), "launches": int(la[q]), "edges": int(ed[q]),
                   "atoms": int(at[q])} for q, name in enumerate(TIMERS)}


def mp_kernel_launches() -> int:
    n = ctypes.c_int64()
    _check(_lib.mp_kernel_launches(ctypes.byref(n)), "mp_kernel_launches")
    return n.value


def mp_head_count(ctx: int) -> int:
    n = ctypes.c_int64()
    _check(_lib.mp_head_count(ctx, ctypes.byref(n)), "mp_head_count")
    return n.value


def mp_head_loss_grad(ctx: int, pos, species, g: int, n_layers: int, e_ref, f_ref,
                      lambda_f: float = 1.0, precision: int = MP_FP32, grad: bool = True):
    """(loss [1] double, grad [n_head] double or None) on the device."""
    loss = torch.empty(1, dtype=torch.float64, device=pos.device)
    gr = (torch.empty(mp_head_count(ctx), dtype=torch.float64, device=pos.device)
          if grad else None)
    _check(_lib.mp_head_loss_grad(ctx, _ptr(pos), _ptr(species), g, n_layers, precision,
                                  _ptr(e_ref), _ptr(f_ref), float(lambda_f), _ptr(loss),
                                  _ptr(gr)), "mp_head_loss_grad")
    return loss, gr


def mp_head_adam_step(ctx: int, grad, lr: float, step: int, beta1: float = 0.9,
                      beta2: float = 0.999, eps: float = 1e-8):
    _check(_lib.mp_head_adam_step(ctx, _ptr(grad), lr, beta1, beta2, eps, step),
           "mp_head_adam_step")


def mp_head_get(ctx: int) -> np.ndarray:
    out = np.zeros(mp_head_count(ctx), dtype=np.float64)
    _check(_lib.mp_head_get(ctx, out.ctypes.data, out.size), "mp_head_get")
    return out


MP_NOALLOC_MAX_ATOMS = 16384 * 2048


def mp_energy_sum_noalloc(e_atom: torch.Tensor, energy: torch.Tensor, n: int | None = None):
    """Sum of the first n per-atom energies (FP64, all of e_atom by default)
    into energy[0] without any device allocation."""
    if e_atom.dtype != torch.float64 or energy.dtype != torch.float64:
        raise ValueError("e_atom and energy must be float64 tensors")
    if energy.numel() < 1:
        raise ValueError("energy needs room for one value")
    n = e_atom.numel() if n is None else int(n)
    if not 0 <= n <= e_atom.numel():
        raise ValueError("n = %d outside 0..%d (the size of e_atom)" % (n, e_atom.numel()))
    _check(_lib.mp_energy_sum_noalloc(_ptr(e_atom), n, _ptr(energy), _stream()),
           "mp_energy_sum_noalloc")


def mp_wait_selftest(ctx: int, max_cycles: int, arrive: bool) -> int:
    """Run the bounded-wait self-test; returns MP_OK or MP_ERR_TIMEOUT."""
    rc = _lib.mp_wait_selftest(ctx, int(max_cycles), 1 if arrive else 0)
    if rc not in (MP_OK, MP_ERR_TIMEOUT):
        _check(rc, "mp_wait_selftest")
    return rc


def mp_strerror(code: int) -> str:
    return _strerror(code)


# ------------------------------------------------------- object wrapper --

class Potential:
    """Owns an mp_ctx for one model on the current CUDA device and stream."""

    def __init__(self, desc, weights: dict):
        self.desc = desc
        self.ctx = mp_create(desc, weights)

    def close(self):
        if self.ctx:
            mp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def energy_forces(self, pos, species, box, n_layers, precision=MP_FP32, n_parts=1,
                      k_hops=None, halo_mode=MP_HALO_GEOM, use_head=False, per_atom=False,
                      part=None):
        """Neighbours, optional partition plan and E/F in one call.  ``part``
        (int32 [n] device, caller order) gives the roots of each of the
        n_parts partitions instead of z slabs; halos are then BFS."""
        mp_set_stream(self.ctx, _stream())
        g = mp_build_neighbors(self.ctx, pos, box)
        plan = None
        try:
            hops = n_layers if k_hops is None else k_hops
            if part is not None:
                plan, _ = mp_partition_assign(self.ctx, g, part, n_parts, hops)
            elif n_parts > 1:
                plan, _ = mp_partition(self.ctx, g, n_parts, hops, halo_mode)
            e_atom = (torch.empty(pos.shape[0], dtype=torch.float64, device=pos.device)
                      if per_atom else None)
            E, F, e_atom = mp_energy_forces(self.ctx, pos, species, g, plan, n_layers, precision,
                                            use_head, e_atom=e_atom)
        finally:
            if plan:
                mp_plan_free(plan)
            mp_graph_free(g)
        return E, F, e_atom

    def energy_forces_stress(self, pos, species, box, n_layers, precision=MP_FP32, n_parts=1,
                             k_hops=None, halo_mode=MP_HALO_GEOM, use_head=False):
        """As energy_forces, plus the 3 x 3 stress (eV/A^3)."""
        mp_set_stream(self.ctx, _stream())
        g = mp_build_neighbors(self.ctx, pos, box)
        plan = None
        try:
            if n_parts > 1:
                plan, _ = mp_partition(self.ctx, g, n_parts,
                                       n_layers if k_hops is None else k_hops, halo_mode)
            E, F, _, S = mp_energy_forces_stress(self.ctx, pos, species, g, plan, n_layers,
                                                 precision, use_head)
        finally:
            if plan:
                mp_plan_free(plan)
            mp_graph_free(g)
        return E, F, S


class EnergyForces(torch.autograd.Function):
    """E(pos) as an autograd node: backward returns -F * grad_output from the
    library's hand-written adjoint (no torch autograd through the network)."""

    @staticmethod
    def forward(ctx, pos, potential, species, box, n_layers, precision):
        E, F, _ = potential.energy_forces(pos.detach(), species, box, n_layers, precision)
        ctx.save_for_backward(F)
        return E[0]

    @staticmethod
    def backward(ctx, grad_out):
        (F,) = ctx.saved_tensors
        return -F.to(torch.float64) * grad_out, None, None, None, None, None
