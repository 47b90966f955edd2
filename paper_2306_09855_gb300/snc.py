"""ctypes binding of libsnc (include/snc.h): argument marshalling only.

Every function of the C ABI is exposed under its own name; the `Network`
class strings them together for a NetworkSpec from `workloads`.  Device
memory for the library comes from PyTorch's caching allocator through the
ABI's allocator callback, and work runs on a PyTorch stream.  The library is
required: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build
from .workloads import DIST_ID, RULE_ID

SNC_OK, SNC_ERR_INVALID_ARG, SNC_ERR_STATE, SNC_ERR_OOM, SNC_ERR_CUDA, SNC_ERR_TIMEOUT, \
    SNC_ERR_UNSUPPORTED = range(7)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "STATE", 3: "OOM", 4: "CUDA", 5: "TIMEOUT",
                6: "UNSUPPORTED"}
SNC_ONE_TO_ONE, SNC_ALL_TO_ALL, SNC_FIXED_INDEGREE, SNC_FIXED_OUTDEGREE, \
    SNC_FIXED_TOTAL_NUMBER, SNC_PAIRWISE_BERNOULLI = range(6)
SNC_DIST_CONST, SNC_DIST_NORMAL = 0, 1


class SncError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status
        self.name = STATUS_NAMES.get(status, str(status))


class snc_range(ctypes.Structure):
    _fields_ = [("first", ctypes.c_uint32), ("n", ctypes.c_uint32)]


class snc_conn_rule(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("allow_autapses", ctypes.c_int32),
                ("allow_multapses", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("k", ctypes.c_uint64), ("p", ctypes.c_double)]


class snc_dist(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("mean", ctypes.c_double), ("std", ctypes.c_double)]


class snc_syn_spec(ctypes.Structure):
    _fields_ = [("weight", snc_dist), ("delay_ms", snc_dist)]


class snc_conn_arrays(ctypes.Structure):
    _fields_ = [("src_ids", ctypes.c_void_p), ("tgt_ids", ctypes.c_void_p), ("weights", ctypes.c_void_p),
                ("delays_ms", ctypes.c_void_p), ("n_conn", ctypes.c_uint64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class snc_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


class snc_config(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("dt_ms", ctypes.c_double), ("device", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("allocator", ctypes.POINTER(snc_allocator))]


class snc_tuning(ctypes.Structure):
    _fields_ = [("sort_digit_bits", ctypes.c_int32), ("sort_group_tiles", ctypes.c_int32),
                ("gen_blocks_per_sm", ctypes.c_int32), ("sort_items", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


class snc_stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_uint64), ("h2d_bytes", ctypes.c_uint64),
                ("d2h_bytes", ctypes.c_uint64), ("n_passes", ctypes.c_int32),
                ("key_bits", ctypes.c_int32), ("device_bytes_peak", ctypes.c_uint64),
                ("source_major", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class snc_conn_view(ctypes.Structure):
    _fields_ = [("n_syn", ctypes.c_uint64), ("n_nodes", ctypes.c_uint64),
                ("n_groups", ctypes.c_uint64), ("row_ptr", ctypes.c_void_p),
                ("target", ctypes.c_void_p), ("delay", ctypes.c_void_p),
                ("weight", ctypes.c_void_p), ("group_ptr", ctypes.c_void_p),
                ("group_first", ctypes.c_void_p)]


class snc_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("device", ctypes.c_int32),
                ("max_slots", ctypes.c_int32), ("batch_max_nets", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("batch_max_syn", ctypes.c_uint64)]


class snc_job_times(ctypes.Structure):
    _fields_ = [("queued_ms", ctypes.c_double), ("build_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("batch_size", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class snc_server_stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint64) for name in (
        "submitted", "completed", "failed", "released", "queued", "running", "builds",
        "batched_builds", "reserved_bytes", "resident_bytes", "peak_reserved_bytes",
        "connections_built")]


SNC_JOB_QUEUED, SNC_JOB_RUNNING, SNC_JOB_DONE, SNC_JOB_FAILED = range(4)

# Every symbol include/snc.h and include/snc_server.h declare.
EXPORTS = ("snc_create", "snc_destroy", "snc_create_population", "snc_connect", "snc_connect_arrays",
           "snc_finalize",
           "snc_synchronize", "snc_get_connections", "snc_copy_connections", "snc_copy_index",
           "snc_copy_network_async",
           "snc_deliver", "snc_set_target_shard", "snc_stage_times",
           "snc_radix_sort_pairs", "snc_radix_sort_pairs_noalloc", "snc_block_sort_pairs", "snc_set_block_sort",
           "snc_get_stats",
           "snc_set_tuning", "snc_get_tuning", "snc_batch_finalize", "snc_batch_finalize_graph",
           "snc_batch_rebuild", "snc_set_wait_test", "snc_set_graph_test", "snc_last_error",
           "snc_server_create", "snc_server_destroy", "snc_server_submit", "snc_server_poll",
           "snc_server_wait_any", "snc_server_context", "snc_server_times", "snc_server_release",
           "snc_server_get_stats", "snc_estimate_build")

_LIB = None


def load(build: bool = True):
    """Load libsnc.so (building it first when missing or stale)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libsnc.so is not built: run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, U32, U64, I32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    sigs = {
        "snc_create": ([ctypes.POINTER(snc_config), ctypes.POINTER(P)], I32),
        "snc_destroy": ([P], I32),
        "snc_create_population": ([P, U32, ctypes.POINTER(U32)], I32),
        "snc_connect": ([P, snc_range, snc_range, ctypes.POINTER(snc_conn_rule),
                         ctypes.POINTER(snc_syn_spec), ctypes.POINTER(U32)], I32),
        "snc_connect_arrays": ([P, snc_range, snc_range, ctypes.POINTER(snc_conn_rule),
                                ctypes.POINTER(snc_syn_spec), ctypes.POINTER(snc_conn_arrays), ctypes.POINTER(U32)],
                               I32),
        "snc_finalize": ([P], I32),
        "snc_batch_finalize": ([ctypes.POINTER(P), I32], I32),
        "snc_batch_finalize_graph": ([ctypes.POINTER(P), I32], I32),
        "snc_batch_rebuild": ([P, ctypes.POINTER(U64), I32], I32),
        "snc_synchronize": ([P], I32),
        "snc_get_connections": ([P, ctypes.POINTER(snc_conn_view)], I32),
        "snc_copy_connections": ([P, P, P, P, P, U64], I32),
        "snc_copy_index": ([P, P, P, P, U64], I32),
        "snc_copy_network_async": ([P, P, P, P, U64, P, P, P, U64], I32),
        "snc_deliver": ([P, P, P, P, U64, P], I32),
        "snc_set_target_shard": ([P, U32, U32], I32),
        "snc_stage_times": ([P, ctypes.POINTER(ctypes.c_float), I32, ctypes.POINTER(I32),
                             ctypes.POINTER(I32)], I32),
        "snc_radix_sort_pairs": ([P, P, P, P, U64, I32, P], I32),
        "snc_radix_sort_pairs_noalloc": ([P, P, P, P, U64, I32, P], I32),
        "snc_block_sort_pairs": ([P, P, U64, I32, U64, P], I32),
        "snc_set_block_sort": ([P, U64], I32),
        "snc_get_stats": ([P, ctypes.POINTER(snc_stats)], I32),
        "snc_set_tuning": ([ctypes.POINTER(snc_tuning)], I32),
        "snc_get_tuning": ([ctypes.POINTER(snc_tuning)], I32),
        "snc_set_wait_test": ([U32, U32], I32),
        "snc_set_graph_test": ([ctypes.c_double, ctypes.c_double, U32], I32),
        "snc_last_error": ([P], ctypes.c_char_p),
        "snc_server_create": ([ctypes.POINTER(snc_server_config), ctypes.POINTER(P)], I32),
        "snc_server_destroy": ([P], I32),
        "snc_server_submit": ([P, P, ctypes.POINTER(U64)], I32),
        "snc_server_poll": ([P, U64, ctypes.POINTER(I32), ctypes.POINTER(snc_conn_view)], I32),
        "snc_server_wait_any": ([P, I32, ctypes.POINTER(U64)], I32),
        "snc_server_context": ([P, U64, ctypes.POINTER(P)], I32),
        "snc_server_times": ([P, U64, ctypes.POINTER(snc_job_times)], I32),
        "snc_server_release": ([P, U64], I32),
        "snc_server_get_stats": ([P, ctypes.POINTER(snc_server_stats)], I32),
        "snc_estimate_build": ([P, ctypes.POINTER(U64), ctypes.POINTER(U64), ctypes.POINTER(U64)], I32),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _LIB = lib
    return lib


def _check(status, ctx=None):
    if status != SNC_OK:
        msg = load().snc_last_error(ctx).decode()
        raise SncError(status, msg)


# ----------------------------------------------------------------------------
# Same-name wrappers of the C ABI.
# ----------------------------------------------------------------------------
def snc_create(cfg):
    h = ctypes.c_void_p()
    _check(load().snc_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def snc_destroy(ctx):
    _check(load().snc_destroy(ctx))


def snc_create_population(ctx, n):
    first = ctypes.c_uint32()
    _check(load().snc_create_population(ctx, n, ctypes.byref(first)), ctx)
    return first.value


def snc_connect(ctx, src, tgt, rule, syn):
    pid = ctypes.c_uint32()
    _check(load().snc_connect(ctx, src, tgt, ctypes.byref(rule), ctypes.byref(syn),
                              ctypes.byref(pid)), ctx)
    return pid.value


def snc_connect_arrays(ctx, src, tgt, rule, syn, src_ids=None, tgt_ids=None, weights=None, delays_ms=None):
    """Connect with explicit node-id arrays and/or per-connection weight and
    delay arrays (host numpy arrays, copied by the library)."""
    keep = []

    def ptr(a, dt):
        if a is None:
            return None, 0
        a = np.ascontiguousarray(a, dtype=dt).ravel()
        buf = a if a.size else np.zeros(1, dt)
        keep.append(buf)
        return buf.ctypes.data, a.size

    sp, _ = ptr(src_ids, np.uint32)
    tp, _ = ptr(tgt_ids, np.uint32)
    wp, nw = ptr(weights, np.float32)
    dp, nd = ptr(delays_ms, np.float32)
    if wp is not None and dp is not None and nw != nd:
        raise ValueError("weights and delays of different lengths")
    arr = snc_conn_arrays(sp, tp, wp, dp, nw if wp is not None else nd)
    pid = ctypes.c_uint32()
    _check(load().snc_connect_arrays(ctx, src, tgt, ctypes.byref(rule), ctypes.byref(syn), ctypes.byref(arr),
                                     ctypes.byref(pid)), ctx)
    return pid.value


def snc_finalize(ctx):
    _check(load().snc_finalize(ctx), ctx)


def snc_batch_finalize(ctxs):
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    _check(load().snc_batch_finalize(arr, len(ctxs)), ctxs[0] if ctxs else None)


def snc_batch_finalize_graph(ctxs):
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    _check(load().snc_batch_finalize_graph(arr, len(ctxs)), ctxs[0] if ctxs else None)


def snc_batch_rebuild(ctx, seeds):
    arr = (ctypes.c_uint64 * len(seeds))(*[int(x) & 0xFFFFFFFFFFFFFFFF for x in seeds])
    _check(load().snc_batch_rebuild(ctx, arr, len(seeds)), ctx)


def snc_synchronize(ctx):
    _check(load().snc_synchronize(ctx), ctx)


def snc_get_connections(ctx):
    v = snc_conn_view()
    _check(load().snc_get_connections(ctx, ctypes.byref(v)), ctx)
    return v


def snc_copy_connections(ctx, n_syn, out=None):
    """Copy the sorted connections into host arrays.  `out` may hold
    preallocated (e.g. page-locked) arrays "src", "tgt" (uint32), "delay"
    (uint16) and "weight" (float32) of at least n_syn entries each."""
    if out is None:
        out = {"src": np.empty(n_syn, np.uint32), "tgt": np.empty(n_syn, np.uint32),
               "delay": np.empty(n_syn, np.uint16), "weight": np.empty(n_syn, np.float32)}
    else:
        want = {"src": np.uint32, "tgt": np.uint32, "delay": np.uint16, "weight": np.float32}
        for name, dt in want.items():
            a = out[name]
            if a.dtype != dt or a.size < n_syn or not a.flags.c_contiguous:
                raise ValueError("output array %r: need %d contiguous %s" % (name, n_syn, np.dtype(dt).name))
    _check(load().snc_copy_connections(ctx, out["src"].ctypes.data, out["tgt"].ctypes.data,
                                       out["delay"].ctypes.data, out["weight"].ctypes.data,
                                       max(n_syn, min(a.size for a in out.values()))), ctx)
    return out


def snc_copy_index(ctx, n_nodes, n_groups, out=None):
    """Copy row_ptr, group_ptr (n_nodes + 1 entries) and group_first
    (n_groups entries) into host uint64 arrays (preallocated in `out` or new)."""
    if out is None:
        out = {"row_ptr": np.empty(n_nodes + 1, np.uint64), "group_ptr": np.empty(n_nodes + 1, np.uint64),
               "group_first": np.empty(max(1, n_groups), np.uint64)}
    for name in ("row_ptr", "group_ptr", "group_first"):
        a = out[name]
        need = n_groups if name == "group_first" else n_nodes + 1
        if a.dtype != np.uint64 or a.size < need or not a.flags.c_contiguous:
            raise ValueError("output array %r: need %d contiguous uint64" % (name, need))
    _check(load().snc_copy_index(ctx, out["row_ptr"].ctypes.data, out["group_ptr"].ctypes.data,
                                 out["group_first"].ctypes.data, out["group_first"].size), ctx)
    return out


def snc_deliver(ctx, src_ptr, grp_ptr, mult_ptr, n_spikes, input_ptr):
    """Deliver a spike array (device pointers: uint32 sources, uint32 group
    indices, float multiplicities) into the float input array of n_nodes."""
    _check(load().snc_deliver(ctx, src_ptr, grp_ptr, mult_ptr, int(n_spikes), input_ptr), ctx)


def snc_set_target_shard(ctx, first, n):
    _check(load().snc_set_target_shard(ctx, int(first), int(n)), ctx)


def snc_stage_times(ctx):
    buf = (ctypes.c_float * 32)()
    ns, npass = ctypes.c_int(), ctypes.c_int()
    _check(load().snc_stage_times(ctx, buf, 32, ctypes.byref(ns), ctypes.byref(npass)), ctx)
    return list(buf[:ns.value]), npass.value


def snc_radix_sort_pairs(keys_in, vals_in, keys_out, vals_out, n, key_bits, stream=0):
    """Device pointers (ints) in, device pointers out."""
    _check(load().snc_radix_sort_pairs(keys_in, vals_in, keys_out, vals_out, n, key_bits,
                                       stream or None))


def snc_radix_sort_pairs_noalloc(keys_in, vals_in, keys_out, vals_out, n, key_bits, stream=0):
    """The same sort without any device allocation (scratch in a static
    device array; n <= SNC_NOALLOC_MAX_PAIRS; calls must not overlap)."""
    _check(load().snc_radix_sort_pairs_noalloc(keys_in, vals_in, keys_out, vals_out, n, key_bits,
                                               stream or None))


SNC_NOALLOC_MAX_PAIRS = 1 << 19


def snc_block_sort_pairs(keys, vals, n, key_bits, block, stream=0):
    """COPASS block sort in place: device pointers (ints) of uint64 keys and
    uint32 values, blocks of `block` pairs (a multiple of 1024)."""
    _check(load().snc_block_sort_pairs(keys, vals, n, key_bits, block, stream or None))


def snc_set_block_sort(ctx, block):
    _check(load().snc_set_block_sort(ctx, int(block)), ctx)


def snc_set_graph_test(bernoulli_sd=10.0, bernoulli_slack=32.0, redraw_rounds=0):
    """Test hook: the bounds graph-recorded builds fix (Bernoulli capacity
    margin, redraw rounds); snc_set_graph_test() restores the defaults."""
    _check(load().snc_set_graph_test(float(bernoulli_sd), float(bernoulli_slack), int(redraw_rounds)))


def snc_set_wait_test(lookback_spin_limit=0, withhold_tile=0xFFFFFFFF):
    """Bound of the sort's look-back waits and a tile that never publishes
    (tests of the TIMEOUT path); snc_set_wait_test() restores the defaults."""
    _check(load().snc_set_wait_test(int(lookback_spin_limit), int(withhold_tile)))


def snc_get_stats(ctx):
    st = snc_stats()
    _check(load().snc_get_stats(ctx, ctypes.byref(st)), ctx)
    return st


def snc_set_tuning(sort_digit_bits=None, sort_group_tiles=None, gen_blocks_per_sm=None, sort_items=None):
    t = snc_get_tuning()
    if sort_digit_bits is not None:
        t.sort_digit_bits = int(sort_digit_bits)
    if sort_group_tiles is not None:
        t.sort_group_tiles = int(sort_group_tiles)
    if gen_blocks_per_sm is not None:
        t.gen_blocks_per_sm = int(gen_blocks_per_sm)
    if sort_items is not None:
        t.sort_items = int(sort_items)
    _check(load().snc_set_tuning(ctypes.byref(t)))
    return t


def snc_get_tuning():
    t = snc_tuning()
    _check(load().snc_get_tuning(ctypes.byref(t)))
    return t


def snc_last_error(ctx=None):
    return load().snc_last_error(ctx).decode()


def snc_estimate_build(ctx):
    """(peak device bytes, resident device bytes, connections) of finalizing ctx."""
    peak, res, n = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().snc_estimate_build(ctx, ctypes.byref(peak), ctypes.byref(res), ctypes.byref(n)), ctx)
    return peak.value, res.value, n.value


def snc_server_create(hbm_budget_bytes, device=0, max_slots=4, batch_max_nets=32, batch_max_syn=40_000_000):
    cfg = snc_server_config(hbm_budget_bytes=int(hbm_budget_bytes), device=int(device),
                            max_slots=int(max_slots), batch_max_nets=int(batch_max_nets), reserved=0,
                            batch_max_syn=int(batch_max_syn))
    h = ctypes.c_void_p()
    _check(load().snc_server_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def snc_server_destroy(srv):
    _check(load().snc_server_destroy(srv))


def snc_server_submit(srv, ctx):
    t = ctypes.c_uint64()
    _check(load().snc_server_submit(srv, ctx, ctypes.byref(t)))
    return t.value


def snc_server_poll(srv, ticket, want_view=False):
    """(state, view or None)."""
    state = ctypes.c_int32()
    v = snc_conn_view()
    _check(load().snc_server_poll(srv, ticket, ctypes.byref(state), ctypes.byref(v) if want_view else None))
    return state.value, (v if want_view and state.value == SNC_JOB_DONE else None)


def snc_server_wait_any(srv, timeout_ms=-1):
    t = ctypes.c_uint64()
    _check(load().snc_server_wait_any(srv, int(timeout_ms), ctypes.byref(t)))
    return t.value


def snc_server_context(srv, ticket):
    h = ctypes.c_void_p()
    _check(load().snc_server_context(srv, ticket, ctypes.byref(h)))
    return h


def snc_server_times(srv, ticket):
    t = snc_job_times()
    _check(load().snc_server_times(srv, ticket, ctypes.byref(t)))
    return t


def snc_server_release(srv, ticket):
    _check(load().snc_server_release(srv, ticket))


def snc_server_get_stats(srv):
    st = snc_server_stats()
    _check(load().snc_server_get_stats(srv, ctypes.byref(st)))
    return st


# ----------------------------------------------------------------------------
# PyTorch as device-memory provider.
# ----------------------------------------------------------------------------
class TorchAllocator:
    """snc_allocator backed by torch's caching allocator on the given device."""

    def __init__(self, device=0):
        import torch
        self._torch = torch
        self.device = device

        def _alloc(nbytes, stream, user):
            try:
                return self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                                stream or 0)
            except Exception:  # the library reports OOM
                return None

        def _free(ptr, nbytes, stream, user):
            self._torch.cuda.caching_allocator_delete(ptr)

        self._alloc_cb = ALLOC_FN(_alloc)
        self._free_cb = FREE_FN(_free)
        self.struct = snc_allocator(self._alloc_cb, self._free_cb, None)


def _rule_struct(pj):
    return snc_conn_rule(kind=RULE_ID[pj.rule], allow_autapses=int(bool(pj.autapses)),
                         allow_multapses=int(bool(pj.multapses)), reserved=0, k=int(pj.k),
                         p=float(pj.p))


def _syn_struct(pj):
    return snc_syn_spec(weight=snc_dist(DIST_ID[pj.weight.kind], 0, float(pj.weight.mean),
                                        float(pj.weight.std)),
                        delay_ms=snc_dist(DIST_ID[pj.delay.kind], 0, float(pj.delay.mean),
                                          float(pj.delay.std)))


def _connect(ctx, pj):
    """snc_connect, or snc_connect_arrays for a projection with explicit
    node-id or per-connection arrays."""
    if getattr(pj, "has_arrays", False):
        return snc_connect_arrays(ctx, snc_range(*pj.src), snc_range(*pj.tgt), _rule_struct(pj), _syn_struct(pj),
                                  src_ids=pj.src_ids, tgt_ids=pj.tgt_ids, weights=pj.weights, delays_ms=pj.delays)
    return snc_connect(ctx, snc_range(*pj.src), snc_range(*pj.tgt), _rule_struct(pj), _syn_struct(pj))


def create_context(spec, device=0, stream_ptr=None, allocator=None):
    """snc_create + CreatePopulation + Connect calls of a NetworkSpec (no finalize)."""
    cfg = snc_config(seed=int(spec.seed) & 0xFFFFFFFFFFFFFFFF, dt_ms=float(spec.dt),
                     device=device, reserved=0, stream=stream_ptr,
                     allocator=ctypes.pointer(allocator) if allocator is not None else None)
    ctx = snc_create(cfg)
    try:
        for n in spec.populations:
            snc_create_population(ctx, int(n))
        for pj in spec.projections:
            _connect(ctx, pj)
    except Exception:
        snc_destroy(ctx)
        raise
    return ctx


class Server:
    """The served form (include/snc_server.h): submit NetworkSpecs, collect
    finished networks, release them.  Device memory comes from the server's
    own pool; results stay on the device until released."""

    def __init__(self, hbm_budget_bytes, device=0, max_slots=4, batch_max_nets=32,
                 batch_max_syn=40_000_000):
        self.device = device
        self.srv = snc_server_create(hbm_budget_bytes, device, max_slots, batch_max_nets, batch_max_syn)

    def submit(self, spec):
        ctx = create_context(spec, self.device)
        try:
            return snc_server_submit(self.srv, ctx)
        except Exception:
            snc_destroy(ctx)
            raise

    def wait_any(self, timeout_ms=-1):
        return snc_server_wait_any(self.srv, timeout_ms)

    def state(self, ticket):
        return snc_server_poll(self.srv, ticket)[0]

    def view(self, ticket):
        return snc_server_poll(self.srv, ticket, want_view=True)[1]

    def times(self, ticket):
        return snc_server_times(self.srv, ticket)

    def to_host(self, ticket):
        """The finished network copied to host numpy arrays (as Network.to_host)."""
        import torch
        ctx = snc_server_context(self.srv, ticket)
        v = self.view(ticket)
        out = snc_copy_connections(ctx, int(v.n_syn))
        t = _view_tensors(v, torch)
        out["row_ptr"] = t["row_ptr"].cpu().numpy()
        out["group_ptr"] = t["group_ptr"].cpu().numpy()
        out["group_first"] = t["group_first"].cpu().numpy()
        out["n_groups"] = int(v.n_groups)
        return out

    def release(self, ticket):
        snc_server_release(self.srv, ticket)

    def stats(self):
        return snc_server_get_stats(self.srv)

    def close(self):
        if self.srv:
            snc_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Network:
    """Create -> Connect -> Finalize -> GetConnections for one NetworkSpec."""

    def __init__(self, spec, device=0, stream=None, allocator="torch", target_shard=None, block_sort=0):
        import torch
        self.spec = spec
        self._torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self._alloc = TorchAllocator(device) if allocator == "torch" else (allocator if allocator else None)
        cfg = snc_config(seed=int(spec.seed) & 0xFFFFFFFFFFFFFFFF, dt_ms=float(spec.dt),
                         device=device, reserved=0, stream=self.stream.cuda_stream,
                         allocator=ctypes.pointer(self._alloc.struct) if self._alloc else None)
        self._cfg = cfg
        self.ctx = snc_create(cfg)
        for n in spec.populations:
            snc_create_population(self.ctx, int(n))
        for pj in spec.projections:
            _connect(self.ctx, pj)
        if target_shard is not None:  # (first, n): keep the connections onto these targets
            snc_set_target_shard(self.ctx, *target_shard)
        if block_sort:  # COPASS block sort with blocks of this many connections
            snc_set_block_sort(self.ctx, block_sort)

    def finalize(self):
        snc_finalize(self.ctx)
        return self

    @staticmethod
    def batch(specs, device=0, stream=None, allocator="torch"):
        """Build several networks with one launch per stage (snc_batch_finalize).

        Returns one Network per spec; each holds a reference to the first
        (whose allocator serves the shared result memory)."""
        nets = [Network(sp, device=device, stream=stream, allocator=allocator) for sp in specs]
        if nets:
            snc_batch_finalize([n.ctx for n in nets])
            for n in nets[1:]:
                n._leader = nets[0]
        return nets

    @staticmethod
    def batch_graph(specs, device=0, stream=None, allocator="torch"):
        """Batched build recorded as a CUDA graph (snc_batch_finalize_graph);
        rebuild() then replays it with new seeds."""
        nets = [Network(sp, device=device, stream=stream, allocator=allocator) for sp in specs]
        if nets:
            snc_batch_finalize_graph([n.ctx for n in nets])
            for n in nets[1:]:
                n._leader = nets[0]
        return nets

    def rebuild(self, seeds):
        """Replay this context's graph build with one seed per member."""
        snc_batch_rebuild(self.ctx, seeds)

    def synchronize(self):
        snc_synchronize(self.ctx)

    def view(self):
        return snc_get_connections(self.ctx)

    def deliver(self, src, grp, mult, input):
        """Deliver a spike array given as device tensors (int32/uint32 sources
        and group indices, float32 multiplicities) into the float32 `input`
        tensor of n_nodes entries (accumulated)."""
        n = int(src.numel())
        if int(grp.numel()) != n or int(mult.numel()) != n:
            raise ValueError("src, grp and mult need the same length")
        for t, size in ((src, 4), (grp, 4), (mult, 4), (input, 4)):
            if not t.is_cuda or t.element_size() != size or not t.is_contiguous():
                raise ValueError("spike arrays and input must be contiguous 4-byte device tensors")
        snc_deliver(self.ctx, src.data_ptr(), grp.data_ptr(), mult.data_ptr(), n, input.data_ptr())

    def tensors(self):
        """Zero-copy torch views of the device arrays."""
        v = self.view()
        return _view_tensors(v, self._torch)

    def to_host(self):
        v = self.view()
        out = snc_copy_connections(self.ctx, int(v.n_syn))
        t = self.tensors()
        out["row_ptr"] = t["row_ptr"].cpu().numpy()
        out["group_ptr"] = t["group_ptr"].cpu().numpy()
        out["group_first"] = t["group_first"].cpu().numpy()
        out["n_groups"] = int(v.n_groups)
        return out

    def to_host_arrays(self, out):
        """Copy the connections into caller-owned host arrays (see
        snc_copy_connections); returns the number of connections."""
        n = int(self.view().n_syn)
        snc_copy_connections(self.ctx, n, out)
        return n

    def to_host_network(self, out, wait=True):
        """Copy the network as it is kept on the device -- target, delay and
        weight arrays plus the CSR and group index (sources implicit in
        row_ptr) -- into caller-owned host arrays (keys "tgt", "delay",
        "weight", "row_ptr", "group_ptr", "group_first"); returns the
        number of connections.  wait=False queues the copies
        (snc_copy_network_async; page-locked arrays) and returns: the arrays
        hold the network after the next synchronize()."""
        v = self.view()
        n = int(v.n_syn)
        cap = min(out[k].size for k in ("tgt", "delay", "weight"))
        if not wait:
            need = {"tgt": (np.uint32, n), "delay": (np.uint16, n), "weight": (np.float32, n),
                    "row_ptr": (np.uint64, int(v.n_nodes) + 1), "group_ptr": (np.uint64, int(v.n_nodes) + 1),
                    "group_first": (np.uint64, int(v.n_groups))}
            for name, (dt, size) in need.items():
                a = out[name]
                if a.dtype != dt or a.size < size or not a.flags.c_contiguous:
                    raise ValueError("output array %r: need %d contiguous %s" % (name, size, np.dtype(dt).name))
            _check(load().snc_copy_network_async(self.ctx, out["tgt"].ctypes.data, out["delay"].ctypes.data,
                                                 out["weight"].ctypes.data, cap, out["row_ptr"].ctypes.data,
                                                 out["group_ptr"].ctypes.data, out["group_first"].ctypes.data,
                                                 out["group_first"].size), self.ctx)
            return n
        _check(load().snc_copy_connections(self.ctx, None, out["tgt"].ctypes.data, out["delay"].ctypes.data,
                                           out["weight"].ctypes.data, cap), self.ctx)
        snc_copy_index(self.ctx, int(v.n_nodes), int(v.n_groups), out)
        return n

    def stage_times(self):
        return snc_stage_times(self.ctx)

    def stats(self):
        return snc_get_stats(self.ctx)

    def close(self):
        if self.ctx:
            snc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _view_tensors(v, torch):
    def dev_tensor(ptr, n, dtype):
        if n == 0:
            return torch.empty(0, dtype=dtype, device="cuda")
        # wrap without copy through the CUDA array interface
        class _Arr:
            pass
        a = _Arr()
        typestr = {torch.uint64: "<u8", torch.int64: "<i8", torch.int32: "<i4",
                   torch.uint32: "<u4", torch.uint16: "<u2", torch.int16: "<i2",
                   torch.float32: "<f4"}[dtype]
        a.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                      "version": 2}
        return torch.as_tensor(a, device="cuda")
    nn = int(v.n_nodes) + 1
    ns = int(v.n_syn)
    ng = int(v.n_groups)
    return {"row_ptr": dev_tensor(v.row_ptr, nn, torch.int64),
            "target": dev_tensor(v.target, ns, torch.int32),
            "delay": dev_tensor(v.delay, ns, torch.int16),
            "weight": dev_tensor(v.weight, ns, torch.float32),
            "group_ptr": dev_tensor(v.group_ptr, nn, torch.int64),
            "group_first": dev_tensor(v.group_first, ng, torch.int64)}
