"""Python binding of the C ABI declared in include/fedfem.h (ctypes).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Each ``fedfem_*`` function here has the name, argument order
and meaning of the C call, takes numpy arrays / Python numbers, and raises
:class:`FedfemError` on a non-zero status.  There is no CPU fallback: if the
shared library is missing, importing this module fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB

if not os.path.exists(LIB):
    raise ImportError(f"libfedfem.so not built ({LIB}); run paper_1909_05098_gb300.build.build()")
_lib = C.CDLL(LIB)

OK, E_ARG, E_MESH, E_STATE, E_UNSTABLE_DT, E_RANGE, E_TIMEOUT, E_CUDA, E_OOM, E_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9
TET4, HEX8 = 4, 8
FP64, FP32_KAHAN, FP32_PLAIN = 0, 1, 2
ORDER_INPUT, ORDER_MORTON, ORDER_RCM = 0, 1, 2
KERNEL_TWO_PHASE, KERNEL_PERSISTENT, KERNEL_TILED, KERNEL_TILED_STAGED, KERNEL_TILED_REP = 0, 1, 2, 3, 4
DOSE_CEM43, DOSE_ARRHENIUS = 0, 1
HEX_ONE_POINT, HEX_FULL = 0, 1
LUMP_ELEMENT, LUMP_UNIFORM = 0, 1

STATUS_NAMES = {0: "OK", -1: "E_ARG", -2: "E_MESH", -3: "E_STATE", -4: "E_UNSTABLE_DT", -5: "E_RANGE",
                -6: "E_TIMEOUT", -7: "E_CUDA", -8: "E_OOM", -9: "E_UNSUPPORTED"}


class FedfemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class fedfem_material(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("T_ref", "rho0", "drho", "c0", "dc", "k0", "dk")]


class fedfem_perfusion(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("w_b", "c_b", "T_a", "Q_m")]


class fedfem_tile(C.Structure):
    _fields_ = [("kernel", C.c_int), ("block", C.c_int), ("tile_nodes", C.c_int), ("blocks_per_sm", C.c_int)]


class fedfem_layout_info(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_elems", C.c_int64), ("n_plain", C.c_int64), ("n_free", C.c_int64),
                ("n_slices", C.c_int64), ("n_gather", C.c_int64), ("max_degree", C.c_int),
                ("tile_nodes", C.c_int), ("n_tiles", C.c_int64), ("n_tile_elems", C.c_int64),
                ("n_halo", C.c_int64), ("max_tile_local", C.c_int), ("max_tile_elems", C.c_int),
                ("max_tile_degree", C.c_int), ("tile_rank_shift", C.c_int)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class fedfem_info(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_elems", C.c_int64), ("n_free", C.c_int64),
                ("n_dirichlet", C.c_int64), ("n_convective", C.c_int64),
                ("elem_type", C.c_int), ("precision", C.c_int), ("order", C.c_int),
                ("dt_cr", C.c_double), ("lambda_max_ref", C.c_double), ("td_scale", C.c_double),
                ("dt_element_bound", C.c_double), ("lanczos_iterations", C.c_int),
                ("steps_done", C.c_int64), ("sim_time", C.c_double), ("device_bytes", C.c_int64),
                ("bytes_per_step", C.c_int64), ("algorithmic_bytes_per_step", C.c_int64),
                ("sm_count", C.c_int), ("grid_blocks", C.c_int), ("block_threads", C.c_int),
                ("kernel", C.c_int), ("tile_nodes", C.c_int), ("lanes", C.c_int)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_ctx_p = C.c_void_p
_i64 = C.c_int64
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)

_SIGS = {
    "fedfem_create": ([C.POINTER(_ctx_p), C.c_int, C.c_int, C.c_void_p], C.c_int),
    "fedfem_set_mesh": ([_ctx_p, C.c_int, _i64, _dp, _i64, _ip], C.c_int),
    "fedfem_set_order": ([_ctx_p, C.c_int], C.c_int),
    "fedfem_set_material": ([_ctx_p, C.POINTER(fedfem_material)], C.c_int),
    "fedfem_set_perfusion": ([_ctx_p, C.POINTER(fedfem_perfusion)], C.c_int),
    "fedfem_set_source": ([_ctx_p, _dp], C.c_int),
    "fedfem_add_gaussian_source": ([_ctx_p, _dp, C.c_double, C.c_double], C.c_int),
    "fedfem_clear_sources": ([_ctx_p], C.c_int),
    "fedfem_set_dirichlet": ([_ctx_p, _i64, _ip, _dp], C.c_int),
    "fedfem_set_convective": ([_ctx_p, _i64, C.c_int, _ip, C.c_double, C.c_double], C.c_int),
    "fedfem_set_nodal_flux": ([_ctx_p, _i64, _ip, _dp], C.c_int),
    "fedfem_precompute": ([_ctx_p, C.c_double, C.c_double, _dp], C.c_int),
    "fedfem_init": ([_ctx_p, _dp, C.c_double], C.c_int),
    "fedfem_init_device": ([_ctx_p, C.c_void_p], C.c_int),
    "fedfem_step": ([_ctx_p, C.c_double, _i64], C.c_int),
    "fedfem_sync": ([_ctx_p, C.POINTER(_i64)], C.c_int),
    "fedfem_read_temperature": ([_ctx_p, _dp], C.c_int),
    "fedfem_read_temperature_device": ([_ctx_p, C.c_void_p], C.c_int),
    "fedfem_get_state": ([_ctx_p, C.c_void_p, C.POINTER(C.c_size_t)], C.c_int),
    "fedfem_set_state": ([_ctx_p, C.c_void_p, C.c_size_t], C.c_int),
    "fedfem_set_tile": ([_ctx_p, C.POINTER(fedfem_tile)], C.c_int),
    "fedfem_get_info": ([_ctx_p, C.POINTER(fedfem_info)], C.c_int),
    "fedfem_last_error": ([_ctx_p], C.c_char_p),
    "fedfem_destroy": ([_ctx_p], None),
    "fedfem_version": ([], C.c_char_p),
    "fedfem_set_hourglass_control": ([_ctx_p, C.c_double], C.c_int),
    "fedfem_set_matrix_free": ([_ctx_p, C.c_int], C.c_int),
    "fedfem_fp64_fma_loop": ([C.c_longlong, C.c_int, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "fedfem_debug_set": ([_ctx_p, C.c_int, _i64], C.c_int),
    "fedfem_plan_layout": ([C.c_int, _i64, _dp, _i64, _ip, _ip, C.c_int, _i64, _ip, _i64, C.c_int, _ip, C.c_int,
                            C.POINTER(fedfem_layout_info)] + [C.c_void_p] * 10, C.c_int),
    "fedfem_set_lanes": ([_ctx_p, C.c_int], C.c_int),
    "fedfem_set_source_schedule": ([_ctx_p, C.c_int, _dp, _dp], C.c_int),
    "fedfem_set_material_table": ([_ctx_p, C.c_int, _dp, _dp, _dp, _dp], C.c_int),
    "fedfem_set_regions": ([_ctx_p, C.c_int, C.POINTER(fedfem_material), C.POINTER(fedfem_perfusion), _ip],
                           C.c_int),
    "fedfem_enable_dose": ([_ctx_p, C.c_int], C.c_int),
    "fedfem_set_dose_model": ([_ctx_p, C.c_int, C.c_double, C.c_double], C.c_int),
    "fedfem_set_hex_integration": ([_ctx_p, C.c_int], C.c_int),
    "fedfem_set_lumping": ([_ctx_p, C.c_int], C.c_int),
    "fedfem_read_dose": ([_ctx_p, _dp], C.c_int),
    "fedfem_read_dose_lane": ([_ctx_p, C.c_int, _dp], C.c_int),
    "fedfem_add_gaussian_source_lane": ([_ctx_p, C.c_int, C.c_int, _dp, C.c_double, C.c_double], C.c_int),
    "fedfem_set_source_lane": ([_ctx_p, C.c_int, _dp], C.c_int),
    "fedfem_read_temperature_lane": ([_ctx_p, C.c_int, _dp], C.c_int),
    "fedfem_set_element_groups": ([_ctx_p, _ip], C.c_int),
    "fedfem_init_lanes_device": ([_ctx_p, C.c_void_p], C.c_int),
    "fedfem_read_lanes_device": ([_ctx_p, C.c_void_p], C.c_int),
    "fedfem_capture_graph": ([_ctx_p, C.c_double, _i64], C.c_int),
    "fedfem_replay_graph": ([_ctx_p], C.c_int),
    "fedfem_mpnn_create": ([C.POINTER(C.c_void_p), C.c_int, _i64, _i64, _ip, _ip, _dp, C.c_double, C.c_int,
                            C.c_int, C.c_void_p], C.c_int),
    "fedfem_mpnn_destroy": ([C.c_void_p], None),
    "fedfem_mpnn_n_params": ([C.c_void_p], _i64),
    "fedfem_mpnn_last_error": ([C.c_void_p], C.c_char_p),
    "fedfem_mpnn_set_params": ([C.c_void_p, C.POINTER(C.c_float)], C.c_int),
    "fedfem_mpnn_get_params": ([C.c_void_p, C.POINTER(C.c_float)], C.c_int),
    "fedfem_mpnn_features": ([C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(fedfem_material),
                              C.c_void_p], C.c_int),
    "fedfem_mpnn_forward": ([C.c_void_p, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "fedfem_mpnn_infer": ([C.c_void_p, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "fedfem_mpnn_sync": ([C.c_void_p], C.c_int),
    "fedfem_mpnn_loss_grad": ([C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_float),
                               C.POINTER(C.c_float)], C.c_int),
    "fedfem_mpnn_adam": ([C.c_void_p, C.c_float], C.c_int),
    "fedfem_gemm_bf16": ([C.c_void_p, _i64, C.c_void_p, _i64, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                          C.c_int, C.c_void_p, _i64, C.c_void_p, C.c_void_p, _i64, C.c_void_p, C.c_void_p,
                          C.c_void_p], C.c_int),
    "fedfem_step_static": ([C.c_int, _i64, _i64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                            C.POINTER(fedfem_material), C.POINTER(fedfem_perfusion), C.c_void_p, C.c_void_p,
                            C.c_double, _i64, C.c_void_p, C.c_void_p], C.c_int),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def library():
    """The loaded ctypes library (for tests that inspect exported symbols)."""
    return _lib


def _check(ctx, rc):
    if rc != OK:
        msg = _lib.fedfem_last_error(ctx).decode() if ctx else ""
        raise FedfemError(rc, msg)


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


# ---- the C calls, same names -------------------------------------------------

def fedfem_version() -> str:
    return _lib.fedfem_version().decode()


def fedfem_fp64_fma_loop(iterations: int, blocks: int, threads: int, sink_dev: int, stream=None):
    """FP64 throughput probe: 16 * iterations * blocks * threads FLOPs on `stream`."""
    rc = _lib.fedfem_fp64_fma_loop(iterations, blocks, threads, C.c_void_p(sink_dev), C.c_void_p(stream))
    if rc != OK:
        raise FedfemError(rc, "fedfem_fp64_fma_loop")


def fedfem_create(device: int = 0, precision: int = FP32_KAHAN, cuda_stream: int | None = None):
    ctx = _ctx_p()
    rc = _lib.fedfem_create(C.byref(ctx), device, precision, C.c_void_p(cuda_stream or 0))
    _check(None, rc)
    return ctx


def fedfem_destroy(ctx):
    _lib.fedfem_destroy(ctx)


def fedfem_set_mesh(ctx, elem_type: int, xyz, conn):
    x, px = _d(xyz)
    c, pc = _i(conn)
    _check(ctx, _lib.fedfem_set_mesh(ctx, elem_type, x.shape[0], px, c.shape[0], pc))


def fedfem_set_order(ctx, order: int):
    _check(ctx, _lib.fedfem_set_order(ctx, order))


def fedfem_set_material(ctx, T_ref, rho0, drho, c0, dc, k0, dk):
    m = fedfem_material(T_ref, rho0, drho, c0, dc, k0, dk)
    _check(ctx, _lib.fedfem_set_material(ctx, C.byref(m)))


def fedfem_set_material_table(ctx, T, rho, c, k):
    arrs = [np.asarray(a, dtype=np.float64).reshape(-1) for a in (T, rho, c, k)]
    if len({a.shape for a in arrs}) != 1:
        raise ValueError("T, rho, c and k differ in length")
    ptrs = [_d(a)[1] for a in arrs]
    _check(ctx, _lib.fedfem_set_material_table(ctx, arrs[0].shape[0], *ptrs))


def fedfem_set_regions(ctx, materials, perfusions, region):
    """materials / perfusions: one per region, objects with the struct's field
    names or tuples in its order; region: one id per element."""
    def mat(m):
        if hasattr(m, "k0"):
            return fedfem_material(m.T_ref, m.rho0, m.drho, m.c0, m.dc, m.k0, m.dk)
        return fedfem_material(*m)

    def perf(p):
        if hasattr(p, "w_b"):
            return fedfem_perfusion(p.w_b, p.c_b, p.T_a, p.Q_m)
        return fedfem_perfusion(*p)

    n = len(materials)
    if len(perfusions) != n:
        raise ValueError("one perfusion per region")
    M = (fedfem_material * n)(*[mat(m) for m in materials])
    P = (fedfem_perfusion * n)(*[perf(p) for p in perfusions])
    r, pr = _i(np.asarray(region).reshape(-1))
    _check(ctx, _lib.fedfem_set_regions(ctx, n, M, P, pr))


def apply_material(ctx, m):
    """Linear laws, or the tabulated ones when the material carries a table."""
    if getattr(m, "table", None) is not None:
        fedfem_set_material_table(ctx, *m.table)
    else:
        fedfem_set_material(ctx, m.T_ref, m.rho0, m.drho, m.c0, m.dc, m.k0, m.dk)


def fedfem_set_perfusion(ctx, w_b, c_b, T_a, Q_m=0.0):
    p = fedfem_perfusion(w_b, c_b, T_a, Q_m)
    _check(ctx, _lib.fedfem_set_perfusion(ctx, C.byref(p)))


def fedfem_set_source(ctx, q_r):
    if q_r is None:
        _check(ctx, _lib.fedfem_set_source(ctx, None))
        return
    q, pq = _d(q_r)
    _check(ctx, _lib.fedfem_set_source(ctx, pq))


def fedfem_add_gaussian_source(ctx, x0, sigma, peak):
    x, px = _d(np.asarray(x0, dtype=np.float64).reshape(3))
    _check(ctx, _lib.fedfem_add_gaussian_source(ctx, px, sigma, peak))


def fedfem_clear_sources(ctx):
    _check(ctx, _lib.fedfem_clear_sources(ctx))


def fedfem_set_dirichlet(ctx, nodes, T):
    n, pn = _i(nodes)
    t, pt = _d(np.broadcast_to(np.asarray(T, dtype=np.float64), n.shape))
    _check(ctx, _lib.fedfem_set_dirichlet(ctx, n.shape[0], pn, pt))


def fedfem_set_convective(ctx, faces, h, T_inf):
    f, pf = _i(faces)
    nverts = f.shape[1] if f.ndim == 2 and f.shape[0] else 3
    _check(ctx, _lib.fedfem_set_convective(ctx, f.shape[0], nverts, pf, h, T_inf))


def fedfem_set_nodal_flux(ctx, nodes, q_W):
    n, pn = _i(nodes)
    q, pq = _d(q_W)
    _check(ctx, _lib.fedfem_set_nodal_flux(ctx, n.shape[0], pn, pq))


def fedfem_precompute(ctx, T_lo, T_hi) -> float:
    out = C.c_double()
    _check(ctx, _lib.fedfem_precompute(ctx, T_lo, T_hi, C.byref(out)))
    return out.value


def fedfem_init(ctx, T0=None, T0_uniform: float = 37.0):
    if T0 is None:
        _check(ctx, _lib.fedfem_init(ctx, None, T0_uniform))
    else:
        t, pt = _d(T0)
        _check(ctx, _lib.fedfem_init(ctx, pt, T0_uniform))


def fedfem_init_device(ctx, T0_dev_ptr: int):
    _check(ctx, _lib.fedfem_init_device(ctx, C.c_void_p(T0_dev_ptr)))


def fedfem_step(ctx, dt: float, n_steps: int):
    _check(ctx, _lib.fedfem_step(ctx, dt, n_steps))


def fedfem_sync(ctx) -> int:
    done = _i64()
    _check(ctx, _lib.fedfem_sync(ctx, C.byref(done)))
    return done.value


def fedfem_sync_status(ctx):
    """(status, steps_done) without raising -- for tests of the error paths."""
    done = _i64()
    rc = _lib.fedfem_sync(ctx, C.byref(done))
    return rc, done.value


def fedfem_read_temperature(ctx, out=None) -> np.ndarray:
    info = fedfem_get_info(ctx)
    if out is None:
        out = np.empty(info["n_nodes"], dtype=np.float64)
    _check(ctx, _lib.fedfem_read_temperature(ctx, out.ctypes.data_as(_dp)))
    return out


def fedfem_read_temperature_device(ctx, out_dev_ptr: int):
    _check(ctx, _lib.fedfem_read_temperature_device(ctx, C.c_void_p(out_dev_ptr)))


def fedfem_get_state(ctx) -> bytes:
    n = C.c_size_t()
    _check(ctx, _lib.fedfem_get_state(ctx, None, C.byref(n)))
    buf = C.create_string_buffer(n.value)
    _check(ctx, _lib.fedfem_get_state(ctx, buf, C.byref(n)))
    return buf.raw[: n.value]


def fedfem_set_state(ctx, state: bytes):
    buf = C.create_string_buffer(state, len(state))
    _check(ctx, _lib.fedfem_set_state(ctx, buf, len(state)))


def fedfem_set_tile(ctx, kernel=KERNEL_PERSISTENT, block=0, tile_nodes=0, blocks_per_sm=0):
    t = fedfem_tile(kernel, block, tile_nodes, blocks_per_sm)
    _check(ctx, _lib.fedfem_set_tile(ctx, C.byref(t)))


def fedfem_get_info(ctx) -> dict:
    info = fedfem_info()
    _check(ctx, _lib.fedfem_get_info(ctx, C.byref(info)))
    return info.as_dict()


def fedfem_last_error(ctx) -> str:
    return _lib.fedfem_last_error(ctx).decode()


def fedfem_debug_set(ctx, key: int, value: int):
    _check(ctx, _lib.fedfem_debug_set(ctx, key, value))


def fedfem_plan_layout(elem_type, xyz, conn, order=ORDER_MORTON, dirichlet_nodes=(), faces=None,
                       tile_nodes=0, groups=None) -> dict:
    """Host-only layout planning (no GPU needed); returns the info dict and arrays."""
    x, px = _d(xyz)
    c, pc = _i(conn)
    if groups is None:
        g, pg = None, None
    else:
        g, pg = _i(groups)
    dn, pdn = _i(np.asarray(dirichlet_nodes, dtype=np.int32).reshape(-1))
    if faces is None or len(faces) == 0:
        fc, pfc, nf, nvf = None, None, 0, 3
    else:
        fc, pfc = _i(faces)
        nf, nvf = fc.shape[0], fc.shape[1]
    info = fedfem_layout_info()
    args = [elem_type, x.shape[0], px, c.shape[0], pc, pg, order, dn.shape[0], pdn, nf, nvf, pfc, tile_nodes,
            C.byref(info)]
    rc = _lib.fedfem_plan_layout(*args, *([None] * 10))
    if rc != OK:
        raise FedfemError(rc, "fedfem_plan_layout")
    d = info.as_dict()
    arrs = {
        "node_of": np.empty(d["n_nodes"], np.int32), "elem_of": np.empty(d["n_elems"], np.int32),
        "slice_off": np.empty(d["n_slices"] + 1, np.int32), "gather": np.empty(d["n_gather"], np.int32),
        "tile_elem_off": np.empty(d["n_tiles"] + 1, np.int32), "tile_elems": np.empty(d["n_tile_elems"], np.int32),
        "tile_lconn": np.empty(d["n_tile_elems"] * elem_type, np.uint16),
        "tile_halo_off": np.empty(d["n_tiles"] + 1, np.int32), "tile_halo": np.empty(d["n_halo"], np.int32),
        "tile_degree": np.empty(d["n_tiles"], np.int32),
    }
    ptrs = [a.ctypes.data_as(C.c_void_p) for a in arrs.values()]
    rc = _lib.fedfem_plan_layout(*args, *ptrs)
    if rc != OK:
        raise FedfemError(rc, "fedfem_plan_layout")
    if d["n_tiles"] == 0:
        for k in list(arrs):
            if k.startswith("tile_"):
                arrs[k] = arrs[k][:0]
    d.update(arrs)
    return d


def fedfem_set_lanes(ctx, n_lanes: int):
    _check(ctx, _lib.fedfem_set_lanes(ctx, n_lanes))


def fedfem_add_gaussian_source_lane(ctx, lane, group, x0, sigma, peak):
    x, px = _d(np.asarray(x0, dtype=np.float64).reshape(3))
    _check(ctx, _lib.fedfem_add_gaussian_source_lane(ctx, lane, group, px, sigma, peak))


def fedfem_set_source_lane(ctx, lane, q_r):
    if q_r is None:
        _check(ctx, _lib.fedfem_set_source_lane(ctx, lane, None))
        return
    q, pq = _d(q_r)
    _check(ctx, _lib.fedfem_set_source_lane(ctx, lane, pq))


def fedfem_read_temperature_lane(ctx, lane: int, out=None) -> np.ndarray:
    info = fedfem_get_info(ctx)
    if out is None:
        out = np.empty(info["n_nodes"], dtype=np.float64)
    _check(ctx, _lib.fedfem_read_temperature_lane(ctx, lane, out.ctypes.data_as(_dp)))
    return out


def fedfem_init_lanes_device(ctx, T0_dev_ptr: int):
    _check(ctx, _lib.fedfem_init_lanes_device(ctx, C.c_void_p(T0_dev_ptr)))


def fedfem_read_lanes_device(ctx, out_dev_ptr: int):
    _check(ctx, _lib.fedfem_read_lanes_device(ctx, C.c_void_p(out_dev_ptr)))


def fedfem_set_element_groups(ctx, groups):
    if groups is None:
        _check(ctx, _lib.fedfem_set_element_groups(ctx, None))
        return
    g, pg = _i(groups)
    _check(ctx, _lib.fedfem_set_element_groups(ctx, pg))


def fedfem_capture_graph(ctx, dt: float, n_steps: int):
    _check(ctx, _lib.fedfem_capture_graph(ctx, dt, n_steps))


def fedfem_replay_graph(ctx):
    _check(ctx, _lib.fedfem_replay_graph(ctx))


def fedfem_step_static(elem_type, n_nodes, n_elems, xyz_dev, conn_dev, row_ptr_dev, slot_dev, material,
                       perfusion, q_r_dev, held_dev, dt, n_steps, T_dev, cuda_stream=0):
    """Allocation-free explicit steps on caller-owned device buffers (raw
    device pointers as ints; q_r_dev / held_dev may be 0).  material and
    perfusion are (T_ref, rho0, drho, c0, dc, k0, dk) and (w_b, c_b, T_a, Q_m)."""
    m = fedfem_material(*material)
    p = fedfem_perfusion(*perfusion)
    rc = _lib.fedfem_step_static(elem_type, n_nodes, n_elems, C.c_void_p(xyz_dev), C.c_void_p(conn_dev),
                                 C.c_void_p(row_ptr_dev), C.c_void_p(slot_dev), C.byref(m), C.byref(p),
                                 C.c_void_p(q_r_dev or 0), C.c_void_p(held_dev or 0), dt, n_steps,
                                 C.c_void_p(T_dev), C.c_void_p(cuda_stream or 0))
    if rc != OK:
        raise FedfemError(rc, "fedfem_step_static")


# ---- convenience wrapper ------------------------------------------------------

def fedfem_set_source_schedule(ctx, t_end, factor):
    e, pe = _d(np.asarray(t_end, dtype=np.float64).reshape(-1))
    f, pf = _d(np.asarray(factor, dtype=np.float64).reshape(-1))
    if e.shape != f.shape:
        raise ValueError("t_end and factor differ in length")
    _check(ctx, _lib.fedfem_set_source_schedule(ctx, e.shape[0], pe, pf))


def fedfem_enable_dose(ctx, on=True):
    _check(ctx, _lib.fedfem_enable_dose(ctx, 1 if on else 0))


def fedfem_set_hex_integration(ctx, rule):
    _check(ctx, _lib.fedfem_set_hex_integration(ctx, int(rule)))


def fedfem_set_hourglass_control(ctx, eps: float):
    _check(ctx, _lib.fedfem_set_hourglass_control(ctx, float(eps)))


def fedfem_set_matrix_free(ctx, on: bool):
    _check(ctx, _lib.fedfem_set_matrix_free(ctx, 1 if on else 0))


def fedfem_set_lumping(ctx, mode):
    _check(ctx, _lib.fedfem_set_lumping(ctx, int(mode)))


def fedfem_set_dose_model(ctx, model, A=0.0, Ea=0.0):
    _check(ctx, _lib.fedfem_set_dose_model(ctx, int(model), float(A), float(Ea)))


def _apply_dose(ctx, dose):
    """dose: False, True / "cem43" (CEM43 minutes) or ("arrhenius", A, Ea)."""
    if not (isinstance(dose, tuple) or dose):
        return
    fedfem_enable_dose(ctx, True)
    if isinstance(dose, tuple):
        if dose[0] != "arrhenius":
            raise ValueError("dose: True, 'cem43' or ('arrhenius', A, Ea)")
        fedfem_set_dose_model(ctx, DOSE_ARRHENIUS, dose[1], dose[2])


def fedfem_read_dose(ctx, lane=0) -> np.ndarray:
    n = fedfem_get_info(ctx)["n_nodes"]
    out = np.empty(n, dtype=np.float64)
    _check(ctx, _lib.fedfem_read_dose_lane(ctx, lane, out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


class Solver:
    """One problem on one GPU: set-up, pre-computation, initial field.

    ``problem`` is any object with the fields of a Pennes problem: elem_type,
    xyz, conn, material (T_ref rho0 drho c0 dc k0 dk), perfusion (w_b c_b T_a
    Q_m), sources (x0 sigma peak), q_r, dirichlet_nodes/_T, conv_faces/_h/
    _T_inf, flux_nodes/_q, T0, T_lo, T_hi."""

    def __init__(self, problem, precision=FP32_KAHAN, device=0, stream=None, order=ORDER_MORTON,
                 kernel=KERNEL_PERSISTENT, T_lo=None, T_hi=None, dose=False, matrix_free=False):
        self.ctx = fedfem_create(device, precision, stream)
        self.problem = problem
        self.dose_model = dose
        self.matrix_free = matrix_free
        if matrix_free and kernel not in (KERNEL_TILED, KERNEL_TILED_STAGED):
            kernel = KERNEL_TILED_STAGED      # the kernels that recompute the element matrices
        try:
            p = problem
            fedfem_set_mesh(self.ctx, p.elem_type, p.xyz, p.conn)
            fedfem_set_order(self.ctx, order)
            if matrix_free:
                fedfem_set_matrix_free(self.ctx, True)
            if getattr(p, "hex_rule", "one-point") == "full":
                fedfem_set_hex_integration(self.ctx, HEX_FULL)
            elif getattr(p, "hex_rule", "one-point") == "hourglass":
                fedfem_set_hourglass_control(self.ctx, p.hourglass_eps)
            if getattr(p, "lumping", "element") == "uniform":
                fedfem_set_lumping(self.ctx, LUMP_UNIFORM)
            apply_material(self.ctx, p.material)
            pf = p.perfusion
            fedfem_set_perfusion(self.ctx, pf.w_b, pf.c_b, pf.T_a, pf.Q_m)
            if getattr(p, "regions", None) is not None:
                fedfem_set_regions(self.ctx, p.region_materials, p.region_perfusion, p.regions)
            for s in p.sources:
                fedfem_add_gaussian_source(self.ctx, s.x0, s.sigma, s.peak)
            if p.q_r is not None:
                fedfem_set_source(self.ctx, p.q_r)
            if len(p.dirichlet_nodes):
                fedfem_set_dirichlet(self.ctx, p.dirichlet_nodes, p.dirichlet_T)
            if len(p.conv_faces):
                fedfem_set_convective(self.ctx, p.conv_faces, p.conv_h, p.conv_T_inf)
            if len(p.flux_nodes):
                fedfem_set_nodal_flux(self.ctx, p.flux_nodes, p.flux_q)
            if len(getattr(p, "schedule_factor", ())):
                fedfem_set_source_schedule(self.ctx, p.schedule_end, p.schedule_factor)
            _apply_dose(self.ctx, dose)
            fedfem_set_tile(self.ctx, kernel)
            self.dt_cr = fedfem_precompute(self.ctx, p.T_lo if T_lo is None else T_lo,
                                           p.T_hi if T_hi is None else T_hi)
            self.init()
        except Exception:
            fedfem_destroy(self.ctx)
            self.ctx = None
            raise

    def init(self, T0=None):
        T0 = self.problem.T0 if T0 is None else T0
        T0 = np.asarray(T0, dtype=np.float64)
        if T0.ndim == 0:
            fedfem_init(self.ctx, None, float(T0))
        else:
            fedfem_init(self.ctx, T0)

    def step(self, dt, n):
        fedfem_step(self.ctx, dt, n)

    def sync(self):
        return fedfem_sync(self.ctx)

    def temperature(self):
        return fedfem_read_temperature(self.ctx)

    def dose(self):
        """CEM43 minutes (or the Arrhenius Omega) per node, input order; needs dose."""
        return fedfem_read_dose(self.ctx)

    def info(self):
        return fedfem_get_info(self.ctx)

    def close(self):
        if self.ctx:
            fedfem_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent planning runs stepped together in ONE context and launch.

    ``meshes`` is a list of lists: each inner list holds 1-4 problems that
    share one mesh (same xyz, conn, material, perfusion, boundary conditions)
    and differ only in their Gaussian sources.  The meshes are concatenated
    (node ids offset), kept apart by element groups, and the scenarios of a
    mesh become scenario lanes; a mesh with fewer than 4 scenarios repeats
    its last one in the unused lanes.  All runs share one dt (the smallest
    critical step) and all materials/perfusion/film parameters must agree."""

    def __init__(self, meshes, precision=FP32_KAHAN, device=0, stream=None, kernel=KERNEL_TILED, schedule=None,
                 dose=False):
        self.meshes = meshes
        first = meshes[0][0]
        xyz, conn, groups, dn, dT = [], [], [], [], []
        self.node_off = [0]
        for g, scen in enumerate(meshes):
            p = scen[0]
            if p.material != first.material or p.perfusion != first.perfusion:
                raise ValueError("all runs of a batch must share material and perfusion")
            if getattr(p, "lumping", "element") != "element" or getattr(p, "hex_rule", "one-point") != "one-point":
                raise ValueError("a batch takes element lumping and the one-point hex rule")
            if (getattr(p, "regions", None) is None) != (getattr(first, "regions", None) is None) or (
                    p.regions is not None and (p.region_materials != first.region_materials
                                               or p.region_perfusion != first.region_perfusion)):
                raise ValueError("all runs of a batch must share the region materials")
            off = self.node_off[-1]
            xyz.append(p.xyz)
            conn.append(np.asarray(p.conn, dtype=np.int64) + off)
            groups.append(np.full(len(p.conn), g, dtype=np.int32))
            dn.append(np.asarray(p.dirichlet_nodes, dtype=np.int64) + off)
            dT.append(np.asarray(p.dirichlet_T, dtype=np.float64))
            self.node_off.append(off + p.n_nodes)
        self.n_nodes = self.node_off[-1]
        self.ctx = fedfem_create(device, precision, stream)
        try:
            fedfem_set_mesh(self.ctx, first.elem_type, np.vstack(xyz), np.vstack(conn))
            fedfem_set_element_groups(self.ctx, np.concatenate(groups))
            fedfem_set_lanes(self.ctx, 4)
            apply_material(self.ctx, first.material)
            pf = first.perfusion
            fedfem_set_perfusion(self.ctx, pf.w_b, pf.c_b, pf.T_a, pf.Q_m)
            if getattr(first, "regions", None) is not None:
                fedfem_set_regions(self.ctx, first.region_materials, first.region_perfusion,
                                   np.concatenate([np.asarray(scen[0].regions) for scen in meshes]))
            fedfem_set_dirichlet(self.ctx, np.concatenate(dn), np.concatenate(dT))
            for g, scen in enumerate(meshes):
                for lane in range(4):
                    p = scen[min(lane, len(scen) - 1)]
                    for s in p.sources:    # restricted to mesh g's nodes (group g)
                        fedfem_add_gaussian_source_lane(self.ctx, lane, g, s.x0, s.sigma, s.peak)
            if schedule is not None:       # (t_end, factor): every run's sources follow it
                fedfem_set_source_schedule(self.ctx, *schedule)
            _apply_dose(self.ctx, dose)
            fedfem_set_tile(self.ctx, kernel)
            self.dt_cr = fedfem_precompute(self.ctx, min(p[0].T_lo for p in meshes),
                                           max(p[0].T_hi for p in meshes))
            fedfem_init(self.ctx, None, float(first.T0))
        except Exception:
            fedfem_destroy(self.ctx)
            self.ctx = None
            raise

    def temperature(self, mesh: int, scenario: int) -> np.ndarray:
        T = fedfem_read_temperature_lane(self.ctx, scenario)
        return T[self.node_off[mesh]: self.node_off[mesh + 1]]

    def dose(self, mesh: int, scenario: int) -> np.ndarray:
        """CEM43 minutes (or the Arrhenius Omega) of one run (needs dose)."""
        D = fedfem_read_dose(self.ctx, scenario)
        return D[self.node_off[mesh]: self.node_off[mesh + 1]]

    def close(self):
        if self.ctx:
            fedfem_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- message-passing surrogate ---------------------------------------------------

def _mcheck(m, rc):
    if rc != OK:
        msg = _lib.fedfem_mpnn_last_error(m).decode() if m else ""
        raise FedfemError(rc, msg)


def fedfem_mpnn_create(n_nodes, src, dst, xyz, length_scale, layers=4, max_batch=1, device=0, cuda_stream=None):
    m = C.c_void_p()
    s, ps = _i(src)
    d, pd = _i(dst)
    x, px = _d(xyz)
    rc = _lib.fedfem_mpnn_create(C.byref(m), device, n_nodes, len(s), ps, pd, px, length_scale, layers, max_batch,
                                 C.c_void_p(cuda_stream or 0))
    _mcheck(None, rc)
    return m


def fedfem_mpnn_destroy(m):
    _lib.fedfem_mpnn_destroy(m)


def fedfem_mpnn_n_params(m) -> int:
    return int(_lib.fedfem_mpnn_n_params(m))


def fedfem_mpnn_set_params(m, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _mcheck(m, _lib.fedfem_mpnn_set_params(m, p.ctypes.data_as(C.POINTER(C.c_float))))


def fedfem_mpnn_get_params(m) -> np.ndarray:
    out = np.empty(fedfem_mpnn_n_params(m), dtype=np.float32)
    _mcheck(m, _lib.fedfem_mpnn_get_params(m, out.ctypes.data_as(C.POINTER(C.c_float))))
    return out


def fedfem_mpnn_features(m, batch, T_dev, q_dev, dirichlet_dev, material, x_dev):
    mat = fedfem_material(*material)
    _mcheck(m, _lib.fedfem_mpnn_features(m, batch, C.c_void_p(T_dev), C.c_void_p(q_dev),
                                         C.c_void_p(dirichlet_dev or 0), C.byref(mat), C.c_void_p(x_dev)))


def fedfem_mpnn_forward(m, batch, x_dev, y_dev):
    _mcheck(m, _lib.fedfem_mpnn_forward(m, batch, C.c_void_p(x_dev), C.c_void_p(y_dev)))


def fedfem_mpnn_infer(m, batch, x_dev, y_dev):
    _mcheck(m, _lib.fedfem_mpnn_infer(m, batch, C.c_void_p(x_dev), C.c_void_p(y_dev)))


def fedfem_mpnn_sync(m):
    _mcheck(m, _lib.fedfem_mpnn_sync(m))


def fedfem_mpnn_loss_grad(m, batch, x_dev, target_dev, mask_dev, want_grad=False):
    loss = C.c_float()
    g = np.empty(fedfem_mpnn_n_params(m), dtype=np.float32) if want_grad else None
    _mcheck(m, _lib.fedfem_mpnn_loss_grad(m, batch, C.c_void_p(x_dev), C.c_void_p(target_dev), C.c_void_p(mask_dev),
                                          C.byref(loss),
                                          g.ctypes.data_as(C.POINTER(C.c_float)) if g is not None else None))
    return loss.value, g


def fedfem_mpnn_adam(m, lr):
    _mcheck(m, _lib.fedfem_mpnn_adam(m, lr))
