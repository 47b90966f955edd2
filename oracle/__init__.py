"""CPU oracle for spiking-network connectivity construction.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg, never by the library.  The arithmetic lives in
snc_oracle.c (plain C, double precision, no CUDA); this module only marshals
numpy arrays through ctypes.

Parity status (see the pins in tests/test_oracle_*.py):
  philox            pinned against cuRAND's host PHILOX4_32_10 generator
  delay_table       pinned against scipy.stats.norm.cdf + chi-square of samples
  binom_table       pinned against scipy.stats.binom.cdf + chi-square of counts
  normal_weight     pinned by closed-form values and a Kolmogorov-Smirnov test
  generate          pinned by brute-force enumeration (one_to_one, all_to_all,
                    the paper's Fig. 1 example), exact per-node counts,
                    autapse/multapse prohibitions, uniformity tests and
                    exhaustive subset-frequency tests on tiny ranges
  build             pinned against numpy's stable lexsort, bincount and a
                    per-source distinct-delay count
  deliver           pinned by the column sums of the weight matrix (every
                    group of every source once), linearity in the
                    multiplicity, a hand-computed example and the group
                    boundaries (tests/test_oracle_deliver.py)
  explicit arrays   node-id arrays pinned to the range forms by renaming
                    invariances, per-connection weights by the Sec. 2.1
                    numbering, delays by hand-computed steps, the complete
                    cases by their unique results (tests/test_oracle_arrays.py)
  copass            the COPASS partition and block sort of Appendix A: pinned
                    by brute force (the left partitions are the first m
                    elements of the stable order), by the block sort equal to
                    numpy's stable argsort, and by planted mistakes
                    (tests/test_oracle_copass.py)
  build_parallel    the same functions on host threads (snc_oracle_par.c):
                    pinned equal, bit for bit, to build() on every rule and
                    flag pair (tests/test_oracle_parallel.py)
"""
from __future__ import annotations

import ctypes
import numpy as np

from .build import build_oracle, build_oracle_par

RULE_ID = {"one_to_one": 0, "all_to_all": 1, "fixed_indegree": 2, "fixed_outdegree": 3,
           "fixed_total_number": 4, "pairwise_bernoulli": 5}
DIST_ID = {"const": 0, "normal": 1}
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "STATE", 3: "OOM", 4: "CUDA", 5: "TIMEOUT",
          6: "UNSUPPORTED"}


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"oracle {what}: {STATUS.get(status, status)}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class _Proj(ctypes.Structure):
    _fields_ = [("src_first", ctypes.c_uint32), ("src_n", ctypes.c_uint32),
                ("tgt_first", ctypes.c_uint32), ("tgt_n", ctypes.c_uint32),
                ("rule", ctypes.c_int32), ("allow_autapses", ctypes.c_int32),
                ("allow_multapses", ctypes.c_int32), ("pad0", ctypes.c_int32),
                ("k", ctypes.c_uint64), ("p", ctypes.c_double),
                ("w_kind", ctypes.c_int32), ("d_kind", ctypes.c_int32),
                ("w_mean", ctypes.c_double), ("w_std", ctypes.c_double),
                ("d_mean", ctypes.c_double), ("d_std", ctypes.c_double),
                ("src_ids", ctypes.c_void_p), ("tgt_ids", ctypes.c_void_p),
                ("w_arr", ctypes.c_void_p), ("d_arr", ctypes.c_void_p),
                ("n_arr", ctypes.c_uint64)]


class _Net(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("dt", ctypes.c_double),
                ("n_nodes", ctypes.c_uint32), ("n_proj", ctypes.c_uint32)]


_LIB = None
_LIB_PAR = None


def _lib_par():
    global _LIB_PAR
    if _LIB_PAR is None:
        _LIB_PAR = ctypes.CDLL(build_oracle_par())
    return _LIB_PAR


def max_threads():
    """Host threads the parallel oracle uses by default."""
    return int(_lib_par().or_max_threads())


def _lib():
    global _LIB
    if _LIB is None:
        _LIB = ctypes.CDLL(build_oracle())
        _LIB.or_normal_weight.restype = ctypes.c_float
    return _LIB


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


def _array(a, dtype, keep):
    """(address, length) of an optional per-projection array as a contiguous
    copy kept alive in `keep`; a given array has a non-null address even
    when it is empty."""
    if a is None:
        return None, 0
    a = np.ascontiguousarray(a, dtype=dtype).ravel()
    buf = a if a.size else np.zeros(1, dtype)
    keep.append(buf)
    return buf.ctypes.data, a.size


class _Marshalled:
    """The ctypes network and projection structs plus the arrays they point into."""

    def __init__(self, spec):
        self.keep = []
        self.net = _Net(seed=int(spec.seed) & 0xFFFFFFFFFFFFFFFF, dt=float(spec.dt),
                        n_nodes=int(spec.n_nodes), n_proj=len(spec.projections))
        self.arr = (_Proj * max(1, len(spec.projections)))()
        for i, pj in enumerate(spec.projections):
            src_ids, ns = _array(getattr(pj, "src_ids", None), np.uint32, self.keep)
            tgt_ids, nt = _array(getattr(pj, "tgt_ids", None), np.uint32, self.keep)
            w_arr, nw = _array(getattr(pj, "weights", None), np.float32, self.keep)
            d_arr, nd = _array(getattr(pj, "delays", None), np.float32, self.keep)
            if src_ids is not None and ns != pj.src[1]:
                raise ValueError("projection %d: src count %d != len(src_ids) %d" % (i, pj.src[1], ns))
            if tgt_ids is not None and nt != pj.tgt[1]:
                raise ValueError("projection %d: tgt count %d != len(tgt_ids) %d" % (i, pj.tgt[1], nt))
            if w_arr is not None and d_arr is not None and nw != nd:
                raise ValueError("projection %d: %d weights but %d delays" % (i, nw, nd))
            self.arr[i] = _Proj(src_first=pj.src[0], src_n=pj.src[1], tgt_first=pj.tgt[0],
                                tgt_n=pj.tgt[1], rule=RULE_ID[pj.rule],
                                allow_autapses=int(bool(pj.autapses)),
                                allow_multapses=int(bool(pj.multapses)), pad0=0, k=int(pj.k),
                                p=float(pj.p), w_kind=DIST_ID[pj.weight.kind],
                                d_kind=DIST_ID[pj.delay.kind], w_mean=float(pj.weight.mean),
                                w_std=float(pj.weight.std), d_mean=float(pj.delay.mean),
                                d_std=float(pj.delay.std), src_ids=src_ids, tgt_ids=tgt_ids,
                                w_arr=w_arr, d_arr=d_arr, n_arr=nw if w_arr is not None else nd)


def _marshal(spec):
    m = _Marshalled(spec)
    return m.net, m.arr, m


def _check(st, what):
    if st != 0:
        raise OracleError(st, what)


def philox(counters, key):
    """Philox4x32-10 of each row of `counters` (n x 4 uint32) under key (k0, k1)."""
    c = np.ascontiguousarray(counters, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(c)
    _lib().or_philox(_ptr(c), ctypes.c_uint32(key[0]), ctypes.c_uint32(key[1]),
                     ctypes.c_uint64(c.shape[0]), _ptr(out))
    return out


def delay_table(mu, sigma, dt):
    """(base, thresholds): step(u) = base + #{T <= u}."""
    thr = np.zeros(16384, dtype=np.uint32)
    base = ctypes.c_uint32(0)
    n = ctypes.c_int(0)
    _check(_lib().or_delay_table(ctypes.c_double(mu), ctypes.c_double(sigma),
                                 ctypes.c_double(dt), _ptr(thr), ctypes.c_int(thr.size),
                                 ctypes.byref(base), ctypes.byref(n)), "delay_table")
    return int(base.value), thr[:n.value].copy()


def binom_table(n, p):
    """(base, thresholds) of Binomial(n, p): count(u) = base + #{T <= u}."""
    thr = np.zeros(16384, dtype=np.uint32)
    base = ctypes.c_uint64(0)
    ln = ctypes.c_int(0)
    _check(_lib().or_binom_table(ctypes.c_uint64(n), ctypes.c_double(p), _ptr(thr),
                                 ctypes.c_int(thr.size), ctypes.byref(base),
                                 ctypes.byref(ln)), "binom_table")
    return int(base.value), thr[:ln.value].copy()


def normal_weight(mu, sigma, w2, w3):
    return float(_lib().or_normal_weight(ctypes.c_double(mu), ctypes.c_double(sigma),
                                         ctypes.c_uint32(w2), ctypes.c_uint32(w3)))


def normal_weights(mu, sigma, w2, w3):
    w2 = np.ascontiguousarray(w2, dtype=np.uint32)
    w3 = np.ascontiguousarray(w3, dtype=np.uint32)
    out = np.empty(w2.size, dtype=np.float32)
    _lib().or_normal_weights(ctypes.c_double(mu), ctypes.c_double(sigma), _ptr(w2), _ptr(w3),
                             ctypes.c_uint64(w2.size), _ptr(out))
    return out


def check_projection(spec, index):
    """Status code Connect gives projection `index` (0 = accepted)."""
    net, arr, _keep = _marshal(spec)
    return int(_lib().or_check_projection(ctypes.byref(net), ctypes.byref(arr[index])))


def count(spec):
    """(total connections, per-projection counts) without storing them."""
    net, arr, _keep = _marshal(spec)
    per = np.zeros(max(1, len(spec.projections)), dtype=np.uint64)
    n = ctypes.c_uint64(0)
    _check(_lib().or_generate(ctypes.byref(net), arr, None, None, None, None,
                              ctypes.c_uint64(0), ctypes.byref(n), _ptr(per)), "count")
    return int(n.value), per[:len(spec.projections)].astype(np.int64)


def generate(spec):
    """All connections in generation order (before the sort)."""
    total, per = count(spec)
    net, arr, _keep = _marshal(spec)
    out = {"src": np.empty(total, np.uint32), "tgt": np.empty(total, np.uint32),
           "delay": np.empty(total, np.uint16), "weight": np.empty(total, np.float32)}
    n = ctypes.c_uint64(0)
    _check(_lib().or_generate(ctypes.byref(net), arr, _ptr(out["src"]), _ptr(out["tgt"]),
                              _ptr(out["delay"]), _ptr(out["weight"]), ctypes.c_uint64(total),
                              ctypes.byref(n), None), "generate")
    out["per_proj"] = per
    return out


def sort_index(n_nodes, src, tgt, delay, weight):
    """Stable sort by (source, delay) and the CSR / group index."""
    src = np.array(src, dtype=np.uint32)
    tgt = np.array(tgt, dtype=np.uint32)
    delay = np.array(delay, dtype=np.uint16)
    weight = np.array(weight, dtype=np.float32)
    n = src.size
    row_ptr = np.zeros(n_nodes + 1, np.uint64)
    group_ptr = np.zeros(n_nodes + 1, np.uint64)
    group_first = np.zeros(max(1, n), np.uint64)
    ng = ctypes.c_uint64(0)
    _check(_lib().or_sort_index(ctypes.c_uint32(n_nodes), ctypes.c_uint64(n), _ptr(src),
                                _ptr(tgt), _ptr(delay), _ptr(weight), _ptr(row_ptr),
                                _ptr(group_ptr), _ptr(group_first), ctypes.byref(ng)),
           "sort_index")
    return {"src": src, "tgt": tgt, "delay": delay, "weight": weight, "row_ptr": row_ptr,
            "group_ptr": group_ptr, "group_first": group_first[:ng.value].copy(),
            "n_groups": int(ng.value)}


def build(spec):
    """The finished network: generate, sort, index."""
    g = generate(spec)
    out = sort_index(spec.n_nodes, g["src"], g["tgt"], g["delay"], g["weight"])
    out["per_proj"] = g["per_proj"]
    return out


def deliver(net, n_nodes, src, grp, mult):
    """Spike delivery through the index of an oracle network (Sec. 2.3):
    per target the exact input (float64), the sum of |weight * mult| and
    the number of additions, and the number of entries naming no group."""
    src = np.ascontiguousarray(src, dtype=np.uint32)
    grp = np.ascontiguousarray(grp, dtype=np.uint32)
    mult = np.ascontiguousarray(mult, dtype=np.float32)
    row_ptr = np.ascontiguousarray(net["row_ptr"], dtype=np.uint64)
    group_ptr = np.ascontiguousarray(net["group_ptr"], dtype=np.uint64)
    group_first = np.ascontiguousarray(net["group_first"], dtype=np.uint64)
    if group_first.size == 0:
        group_first = np.zeros(1, np.uint64)
    tgt = np.ascontiguousarray(net["tgt"], dtype=np.uint32)
    weight = np.ascontiguousarray(net["weight"], dtype=np.float32)
    inp = np.zeros(max(1, n_nodes), np.float64)
    absv = np.zeros(max(1, n_nodes), np.float64)
    terms = np.zeros(max(1, n_nodes), np.uint64)
    bad = ctypes.c_uint64(0)
    _check(_lib().or_deliver(ctypes.c_uint32(n_nodes), ctypes.c_uint64(tgt.size), _ptr(row_ptr), _ptr(group_ptr),
                             _ptr(group_first), _ptr(tgt), _ptr(weight), ctypes.c_uint64(src.size), _ptr(src),
                             _ptr(grp), _ptr(mult), _ptr(inp), _ptr(absv), _ptr(terms), ctypes.byref(bad)),
           "deliver")
    return {"input": inp[:n_nodes], "abs": absv[:n_nodes], "terms": terms[:n_nodes], "bad": int(bad.value)}


def generate_primary(spec, proj, primary):
    """Connections of one primary node of projection `proj`, in slot order."""
    net, arr, _keep = _marshal(spec)
    pj = spec.projections[proj]
    cap = max(1, int(pj.src[1]) + int(pj.tgt[1]) + int(pj.k) + 1)
    out = {"src": np.empty(cap, np.uint32), "tgt": np.empty(cap, np.uint32),
           "delay": np.empty(cap, np.uint16), "weight": np.empty(cap, np.float32)}
    n = ctypes.c_uint64(0)
    _check(_lib().or_generate_primary(ctypes.byref(net), arr, ctypes.c_uint32(proj),
                                      ctypes.c_uint32(primary), _ptr(out["src"]),
                                      _ptr(out["tgt"]), _ptr(out["delay"]),
                                      _ptr(out["weight"]), ctypes.c_uint64(cap),
                                      ctypes.byref(n)), "generate_primary")
    return {k: v[:n.value].copy() for k, v in out.items()}


def generate_parallel(spec, threads=0):
    """generate() on host threads: the same arrays (threads = 0: all)."""
    net, arr, _keep = _marshal(spec)
    lib = _lib_par()
    per = np.zeros(max(1, len(spec.projections)), dtype=np.uint64)
    n = ctypes.c_uint64(0)
    _check(lib.or_generate_par(ctypes.byref(net), arr, None, None, None, None, ctypes.c_uint64(0),
                               ctypes.byref(n), _ptr(per), ctypes.c_int(threads)), "count")
    total = int(n.value)
    out = {"src": np.empty(total, np.uint32), "tgt": np.empty(total, np.uint32),
           "delay": np.empty(total, np.uint16), "weight": np.empty(total, np.float32)}
    _check(lib.or_generate_par(ctypes.byref(net), arr, _ptr(out["src"]), _ptr(out["tgt"]), _ptr(out["delay"]),
                               _ptr(out["weight"]), ctypes.c_uint64(total), ctypes.byref(n), None,
                               ctypes.c_int(threads)), "generate")
    out["per_proj"] = per[:len(spec.projections)].astype(np.int64)
    return out


def build_parallel(spec, threads=0):
    """build() on host threads: the same network, bit for bit."""
    g = generate_parallel(spec, threads)
    n_nodes = spec.n_nodes
    n = g["src"].size
    row_ptr = np.zeros(n_nodes + 1, np.uint64)
    group_ptr = np.zeros(n_nodes + 1, np.uint64)
    group_first = np.zeros(max(1, n), np.uint64)
    ng = ctypes.c_uint64(0)
    _check(_lib_par().or_sort_index_par(ctypes.c_uint32(n_nodes), ctypes.c_uint64(n), _ptr(g["src"]),
                                        _ptr(g["tgt"]), _ptr(g["delay"]), _ptr(g["weight"]), _ptr(row_ptr),
                                        _ptr(group_ptr), _ptr(group_first), ctypes.byref(ng),
                                        ctypes.c_int(threads)), "sort_index")
    return {"src": g["src"], "tgt": g["tgt"], "delay": g["delay"], "weight": g["weight"], "row_ptr": row_ptr,
            "group_ptr": group_ptr, "group_first": group_first[:ng.value], "n_groups": int(ng.value),
            "per_proj": g["per_proj"]}


def copass_partition(runs, m):
    """Left-partition sizes of the COPASS partition (Appendix A) of sorted
    uint64 runs with sum = m."""
    runs = [np.ascontiguousarray(r, dtype=np.uint64) for r in runs]
    k = len(runs)
    bufs = [r if r.size else np.zeros(1, np.uint64) for r in runs]
    ptrs = (ctypes.c_void_p * max(1, k))(*[b.ctypes.data for b in bufs])
    lens = np.array([r.size for r in runs] or [0], dtype=np.uint64)
    part = np.zeros(max(1, k), dtype=np.uint64)
    _check(_lib().or_copass_partition(ptrs, _ptr(lens), ctypes.c_uint32(k), ctypes.c_uint64(int(m)),
                                      _ptr(part)), "copass_partition")
    return part[:k].astype(np.int64)


def copass_sort(keys, vals, block):
    """The COPASS block sort (Appendix A) of uint64 keys with uint64 values,
    blocks of `block` elements: (sorted keys, values)."""
    keys = np.array(keys, dtype=np.uint64)
    vals = np.array(vals, dtype=np.uint64)
    _check(_lib().or_copass_sort(_ptr(keys), _ptr(vals), ctypes.c_uint64(keys.size), ctypes.c_uint64(int(block))),
           "copass_sort")
    return keys, vals
