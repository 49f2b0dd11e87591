"""Python binding of libvc (include/vc.h): exact vertex cover on a GB300 GPU.

Argument marshalling only: every step of the search runs in the CUDA kernels of ``libvc.so``.
Graphs are CSR arrays (``offsets`` n+1, ``neighbors`` 2m, int32) given as numpy arrays (host) or
torch CUDA tensors (device).  If ``libvc.so`` has not been built, importing a solver raises; there
is no CPU fallback.

    mvc(offsets, neighbors)            -> Answer(size, cover, stats)
    pvc(offsets, neighbors, k)         -> Answer(found, cover, stats)
    mvc_batch(batch)                   -> (sizes, covers, stats)
    greedy(offsets, neighbors)         -> (size, cover)
    reduce_node(offsets, neighbors, deg, S, m, problem, bound, rules) -> (deg, S, m, pruned)
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvc.so")

VC_OK, VC_EINVAL, VC_ENOMEM, VC_ETIMEOUT, VC_ESTACK, VC_ECUDA, VC_ECANCELLED = 0, -1, -2, -3, -4, -5, -6
MVC, PVC = 0, 1
RULE_DEG1, RULE_DEG2TRI, RULE_HIGH, RULE_ALL = 1, 2, 4, 7

EXPORTED = ["vc_mvc", "vc_pvc", "vc_mvc_batch", "vc_greedy", "vc_reduce_node", "vc_last_sm_nodes",
            "vc_release", "vc_strerror", "vc_version", "vc_mvc_noalloc",
            "vc_server_create", "vc_server_submit", "vc_server_poll", "vc_server_release", "vc_server_drain",
            "vc_server_stats", "vc_server_destroy", "vc_plan_create_mvc_batch", "vc_plan_launch", "vc_plan_results",
            "vc_plan_completion_ns", "vc_plan_destroy", "vc_l2_copy_probe"]
NOALLOC_MAX_N = 512


class VCError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where} failed: {_strerror(code)} ({code})")


class Graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("offsets", ctypes.c_void_p), ("neighbors", ctypes.c_void_p),
                ("on_device", ctypes.c_int32)]


class Config(ctypes.Structure):
    _fields_ = [("worker_threads", ctypes.c_int32), ("num_workers", ctypes.c_int32),
                ("width", ctypes.c_int32), ("worklist_capacity", ctypes.c_int32),
                ("donate_threshold", ctypes.c_float), ("idle_timeout_ns", ctypes.c_int64),
                ("skip_validation", ctypes.c_int32), ("stage_csr", ctypes.c_int32),
                ("cancel", ctypes.c_void_p), ("node_in_global", ctypes.c_int32), ("bit_rows", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("nodes_visited", ctypes.c_int64), ("stack_pushes", ctypes.c_int64),
                ("stack_pops", ctypes.c_int64), ("donations", ctypes.c_int64),
                ("worklist_pops", ctypes.c_int64), ("rule_passes", ctypes.c_int64),
                ("csr_words", ctypes.c_int64), ("entry_bytes_moved", ctypes.c_int64),
                ("max_depth", ctypes.c_int32), ("greedy_ub", ctypes.c_int32), ("workers", ctypes.c_int32),
                ("worker_threads", ctypes.c_int32), ("width", ctypes.c_int32), ("csr_staged", ctypes.c_int32),
                ("status", ctypes.c_int32),
                ("kernel_ms", ctypes.c_float), ("total_ms", ctypes.c_float),
                ("trace_ns", ctypes.c_int64 * 4), ("idle_polls", ctypes.c_int64),
                ("node_in_global", ctypes.c_int32), ("stack_depth", ctypes.c_int32),
                ("bit_rows", ctypes.c_int32), ("trace_cycles", ctypes.c_int64 * 16)]

    def as_dict(self) -> dict:
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["trace_ns"] = list(self.trace_ns)
        d["trace_cycles"] = list(self.trace_cycles)
        return d


class RequestInfo(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int32), ("answer", ctypes.c_int32), ("status", ctypes.c_int32),
                ("greedy", ctypes.c_int32), ("submit_ns", ctypes.c_int64), ("admit_ns", ctypes.c_int64),
                ("done_ns", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class ServerCounters(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("pending", ctypes.c_int64), ("in_flight", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("epochs", ctypes.c_int64), ("nodes_visited", ctypes.c_int64),
                ("workers", ctypes.c_int32), ("worker_threads", ctypes.c_int32),
                ("slots_per_epoch", ctypes.c_int32), ("arena_bytes", ctypes.c_int64), ("records", ctypes.c_int64),
                ("classes", ctypes.c_int32), ("small_max_n", ctypes.c_int32), ("small_workers", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None
_lib_path = None


def library_path() -> str:
    return LIB_PATH


def load(path: str | None = None):
    """Loads libvc.so (raising if it is missing) and declares the C signatures.  ``path`` selects
    another build of the library (an instrumented variant, see build.build_variant); a process
    loads one library only."""
    global _lib, _lib_path
    if _lib is not None:
        if path is not None and os.path.abspath(path) != _lib_path:
            raise RuntimeError(f"{_lib_path} is already loaded in this process; cannot also load {path}")
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libvc.so not built at {path}; run python -m paper_2204_10402_gb300.build")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    gp, cp, sp = ctypes.POINTER(Graph), ctypes.POINTER(Config), ctypes.POINTER(Stats)
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.vc_mvc.argtypes = [gp, cp, P, P, i32p, sp]
    lib.vc_pvc.argtypes = [gp, i32, cp, P, i32p, P, i32p, sp]
    lib.vc_mvc_batch.argtypes = [i32, P, P, P, P, i32, cp, P, P, P, sp]
    lib.vc_greedy.argtypes = [gp, cp, P, P, i32p]
    lib.vc_reduce_node.argtypes = [gp, P, i32p, i32p, i32, i32, i32, i32, cp, P, i32p]
    lib.vc_last_sm_nodes.argtypes = [P, i32]
    lib.vc_mvc_noalloc.argtypes = [gp, cp, P, P, i32p, sp]
    lib.vc_server_create.argtypes = [cp, ctypes.c_size_t, i32, ctypes.POINTER(ctypes.c_void_p)]
    lib.vc_server_submit.argtypes = [P, gp, i32, i32, ctypes.POINTER(ctypes.c_uint64)]
    lib.vc_server_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(RequestInfo)]
    lib.vc_server_release.argtypes = [P, ctypes.c_uint64]
    lib.vc_server_drain.argtypes = [P, i64]
    lib.vc_server_stats.argtypes = [P, ctypes.POINTER(ServerCounters)]
    lib.vc_server_destroy.argtypes = [P]
    lib.vc_plan_create_mvc_batch.argtypes = [i32, P, P, P, P, i32, cp, ctypes.POINTER(ctypes.c_void_p)]
    lib.vc_plan_launch.argtypes = [P, P]
    lib.vc_plan_results.argtypes = [P, P, P, P, i32, sp]
    lib.vc_plan_completion_ns.argtypes = [P, P, P]
    lib.vc_plan_destroy.argtypes = [P]
    lib.vc_l2_copy_probe.argtypes = [P, P, ctypes.c_size_t, i32, P]
    lib.vc_release.argtypes = []
    lib.vc_strerror.argtypes = [ctypes.c_int]
    lib.vc_strerror.restype = ctypes.c_char_p
    lib.vc_version.argtypes = []
    for name in ("vc_mvc", "vc_pvc", "vc_mvc_batch", "vc_greedy", "vc_reduce_node", "vc_last_sm_nodes",
                 "vc_release", "vc_version", "vc_mvc_noalloc", "vc_server_create", "vc_server_submit",
                 "vc_server_poll", "vc_server_release", "vc_server_drain", "vc_server_stats", "vc_server_destroy",
                 "vc_plan_create_mvc_batch", "vc_plan_launch", "vc_plan_results", "vc_plan_completion_ns",
                 "vc_plan_destroy"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    _lib_path = os.path.abspath(path)
    return lib


def _strerror(code: int) -> str:
    try:
        return load().vc_strerror(code).decode()
    except Exception:
        return str(code)


def _check(rc: int, where: str):
    if rc != VC_OK:
        raise VCError(rc, where)


# ---------------------------------------------------------------------------------------------
# argument marshalling
# ---------------------------------------------------------------------------------------------

def _is_cuda_tensor(x) -> bool:
    return hasattr(x, "is_cuda") and bool(getattr(x, "is_cuda"))


def _host_i32(x) -> np.ndarray:
    """A host int32 copy (or view) of an integer array; values outside int32 are an error, not a
    silent wrap."""
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    a = np.asarray(x)
    if a.size and not np.issubdtype(a.dtype, np.integer):
        raise TypeError(f"CSR arrays must hold integers, not {a.dtype}")
    if a.dtype != np.int32 and a.size and (int(a.min()) < -2**31 or int(a.max()) >= 2**31):
        raise ValueError("CSR values do not fit int32")
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(x) -> int:
    if _is_cuda_tensor(x):
        return int(x.data_ptr())
    return int(x.ctypes.data)


def _stream(stream) -> int:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return int(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return 0
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


def make_config(**kw) -> Config:
    c = Config()
    for k, v in kw.items():
        if v is None:
            continue
        if k == "cancel":
            c.cancel = v
        else:
            setattr(c, k, v)
    return c


def _device_csr(offsets, neighbors):
    """Contiguous int32 CUDA tensors of a CSR on the current device, which the library launches on.
    The caller keeps them alive until the library call has returned."""
    import torch
    if not _is_cuda_tensor(neighbors) or neighbors.device != offsets.device:
        raise ValueError("offsets and neighbors must be CUDA tensors on the same device")
    if offsets.device.index != torch.cuda.current_device():
        raise ValueError(f"the CSR is on {offsets.device} but the current device is "
                         f"cuda:{torch.cuda.current_device()}; call under torch.cuda.device({offsets.device})")
    if offsets.dtype != torch.int32 or neighbors.dtype != torch.int32:
        raise TypeError("CSR tensors must be int32")
    off = offsets.contiguous()
    nb = neighbors.contiguous() if neighbors.numel() > 0 else torch.zeros(1, dtype=torch.int32, device=offsets.device)
    return off, nb


def _graph(offsets, neighbors):
    """Returns (Graph, keepalive) for host numpy or CUDA tensor CSR arrays."""
    if _is_cuda_tensor(offsets):
        off, nb = _device_csr(offsets, neighbors)
        return Graph(off.numel() - 1, off.data_ptr(), nb.data_ptr(), 1), (off, nb)
    off = _host_i32(offsets)
    nbr = _host_i32(neighbors)
    if nbr.size == 0:
        nbr = np.zeros(1, dtype=np.int32)
    return Graph(off.size - 1, off.ctypes.data, nbr.ctypes.data, 0), (off, nbr)


def _cover_buffer(g: Graph, like):
    if g.on_device:
        import torch
        return torch.empty(max(g.n, 1), dtype=torch.int32, device=like.device)
    return np.zeros(max(g.n, 1), dtype=np.int32)


@dataclass
class Answer:
    value: int          # MVC: minimum size; PVC: 1 if a cover of size <= k exists
    cover: object       # 0/1 mask (numpy array, or torch tensor for device inputs), None if none
    cover_size: int
    stats: dict


def mvc(offsets, neighbors, config: Config | None = None, stream=None, want_cover: bool = True) -> Answer:
    """Minimum vertex cover (Sec. II-A) of one graph."""
    lib = load()
    g, keep = _graph(offsets, neighbors)
    cover = _cover_buffer(g, offsets) if want_cover else None
    size = ctypes.c_int32(-1)
    st = Stats()
    rc = lib.vc_mvc(ctypes.byref(g), ctypes.byref(config) if config else None, _stream(stream),
                    _ptr(cover) if cover is not None else None, ctypes.byref(size), ctypes.byref(st))
    _check(rc, "vc_mvc")
    if cover is not None:
        cover = cover[: g.n]
    return Answer(int(size.value), cover, int(size.value), st.as_dict())


def mvc_noalloc(offsets, neighbors, config: Config | None = None, stream=None) -> Answer:
    """MVC of one small graph (n <= 512) whose CSR is on the device, with no memory allocation by
    the library: for callers whose device memory is owned by a pool or arena, or whose request
    path must not call cudaMalloc/cudaFree.  The cover comes back as a device tensor allocated
    here by torch, outside the library call."""
    import torch
    lib = load()
    g, keep = _graph(offsets, neighbors)
    if not g.on_device:
        raise ValueError("mvc_noalloc takes CUDA tensors")
    cover = torch.empty(max(g.n, 1), dtype=torch.int32, device=offsets.device)
    size = ctypes.c_int32(-1)
    st = Stats()
    rc = lib.vc_mvc_noalloc(ctypes.byref(g), ctypes.byref(config) if config else None, _stream(stream),
                            cover.data_ptr(), ctypes.byref(size), ctypes.byref(st))
    _check(rc, "vc_mvc_noalloc")
    return Answer(int(size.value), cover[: g.n], int(size.value), st.as_dict())


def pvc(offsets, neighbors, k: int, config: Config | None = None, stream=None, want_cover: bool = True) -> Answer:
    """Parameterized vertex cover (Sec. II-A): is there a cover of size <= k?"""
    lib = load()
    g, keep = _graph(offsets, neighbors)
    cover = _cover_buffer(g, offsets) if want_cover else None
    found = ctypes.c_int32(0)
    csize = ctypes.c_int32(-1)
    st = Stats()
    rc = lib.vc_pvc(ctypes.byref(g), int(k), ctypes.byref(config) if config else None, _stream(stream),
                    ctypes.byref(found), _ptr(cover) if cover is not None else None, ctypes.byref(csize),
                    ctypes.byref(st))
    _check(rc, "vc_pvc")
    if cover is not None:
        cover = cover[: g.n] if found.value else None
    return Answer(int(found.value), cover, int(csize.value), st.as_dict())


def mvc_batch(vtx, edge, offsets, neighbors, config: Config | None = None, stream=None,
              want_covers: bool = True):
    """Batched MVC over packed graphs (see graphs.pack for the layout).  ``vtx`` and ``edge`` are
    host arrays of G+1 prefix sums; ``offsets``/``neighbors`` host arrays or CUDA tensors."""
    lib = load()
    vtx = _host_i32(vtx)
    edge = _host_i32(edge)
    G = vtx.size - 1
    on_dev = _is_cuda_tensor(offsets)
    if on_dev:
        import torch
        off_t, nb_t = _device_csr(offsets, neighbors)
        off_p, nb_p = off_t.data_ptr(), nb_t.data_ptr()
        covers = torch.empty(max(int(vtx[-1]), 1), dtype=torch.int32, device=offsets.device) if want_covers else None
    else:
        off_t = _host_i32(offsets)
        nb_t = _host_i32(neighbors)
        if nb_t.size == 0:
            nb_t = np.zeros(1, dtype=np.int32)
        off_p, nb_p = off_t.ctypes.data, nb_t.ctypes.data
        covers = np.zeros(max(int(vtx[-1]), 1), dtype=np.int32) if want_covers else None
    sizes = np.zeros(max(G, 1), dtype=np.int32)
    st = Stats()
    rc = lib.vc_mvc_batch(G, vtx.ctypes.data, edge.ctypes.data, off_p, nb_p, 1 if on_dev else 0,
                          ctypes.byref(config) if config else None, _stream(stream), sizes.ctypes.data,
                          _ptr(covers) if covers is not None else None, ctypes.byref(st))
    _check(rc, "vc_mvc_batch")
    return sizes[:G], covers, st.as_dict()


def greedy(offsets, neighbors, config: Config | None = None, stream=None):
    """Greedy upper bound of Sec. II-B computed on the GPU."""
    lib = load()
    g, keep = _graph(offsets, neighbors)
    cover = _cover_buffer(g, offsets)
    size = ctypes.c_int32(-1)
    rc = lib.vc_greedy(ctypes.byref(g), ctypes.byref(config) if config else None, _stream(stream), _ptr(cover),
                       ctypes.byref(size))
    _check(rc, "vc_greedy")
    return int(size.value), cover[: g.n]


def reduce_node(offsets, neighbors, deg, S: int, m: int, problem: int, bound: int, rules: int = RULE_ALL,
                config: Config | None = None, stream=None, branch: int = -1):
    """One tree node's fixpoint reduction on the GPU (rule tests).  branch = v >= 0 (or -2-v) puts v
    (or N(v)) into S first, treating ``deg`` as a fixpoint, as the traversal does for a child."""
    lib = load()
    g, keep = _graph(offsets, neighbors)
    if g.on_device:
        import torch
        d = deg.to(dtype=torch.int32).contiguous().clone()
    else:
        d = np.array(deg, dtype=np.int32).copy()
        if d.size == 0:
            d = np.zeros(1, dtype=np.int32)
    s = ctypes.c_int32(S)
    mm = ctypes.c_int32(m)
    pruned = ctypes.c_int32(0)
    rc = lib.vc_reduce_node(ctypes.byref(g), _ptr(d), ctypes.byref(s), ctypes.byref(mm), int(problem), int(bound),
                            int(rules), int(branch), ctypes.byref(config) if config else None, _stream(stream),
                            ctypes.byref(pruned))
    _check(rc, "vc_reduce_node")
    return d[: g.n], int(s.value), int(mm.value), bool(pruned.value)


def last_sm_nodes() -> np.ndarray:
    """Search-tree nodes expanded per SM by the last traversal (Sec. V-C load measure)."""
    lib = load()
    buf = np.zeros(1024, dtype=np.int64)
    rc = lib.vc_last_sm_nodes(buf.ctypes.data, buf.size)
    if rc < 0:
        raise VCError(rc, "vc_last_sm_nodes")
    return buf[:rc].copy()


def l2_copy_probe(dst, src, passes: int, stream=None):
    """Copies CUDA tensor src onto dst `passes` times in one launch through L2 (measurement
    helper; see vc_l2_copy_probe).  Returns without waiting for the stream."""
    if not (_is_cuda_tensor(dst) and _is_cuda_tensor(src)) or dst.numel() * dst.element_size() != src.numel() * src.element_size():
        raise ValueError("l2_copy_probe takes two CUDA tensors of the same size in bytes")
    _check(load().vc_l2_copy_probe(dst.data_ptr(), src.data_ptr(), src.numel() * src.element_size(), int(passes),
                                   _stream(stream)), "vc_l2_copy_probe")


def release():
    _check(load().vc_release(), "vc_release")


class Server:
    """Serving with continuous batching (include/vc_server.h): one persistent launch searches all
    admitted requests at once; requests submitted while it runs join it.

        with Server(max_n=3000) as srv:
            rid = srv.submit(offsets, neighbors, MVC)
            srv.drain()
            srv.poll(rid)["answer"]
    """

    def __init__(self, max_n: int, budget_bytes: int = 0, config: Config | None = None):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.vc_server_create(ctypes.byref(config) if config else None, int(budget_bytes), int(max_n),
                                    ctypes.byref(h)), "vc_server_create")
        self._h = h
        self._lib = lib

    def submit(self, offsets, neighbors, kind: int, k: int = 0) -> int:
        g, keep = _graph(offsets, neighbors)
        if g.on_device:
            raise ValueError("Server.submit takes host arrays")
        rid = ctypes.c_uint64(0)
        _check(self._lib.vc_server_submit(self._h, ctypes.byref(g), int(kind), int(k), ctypes.byref(rid)),
               "vc_server_submit")
        return int(rid.value)

    def poll(self, rid: int, release: bool = False) -> dict:
        """The request's state; with release=True a finished request is also forgotten."""
        info = RequestInfo()
        _check(self._lib.vc_server_poll(self._h, ctypes.c_uint64(rid), ctypes.byref(info)), "vc_server_poll")
        if release and info.done:
            self.release(rid)
        return info.as_dict()

    def release(self, rid: int):
        _check(self._lib.vc_server_release(self._h, ctypes.c_uint64(rid)), "vc_server_release")

    def drain(self, timeout_ms: int = 0):
        _check(self._lib.vc_server_drain(self._h, int(timeout_ms)), "vc_server_drain")

    def stats(self) -> dict:
        c = ServerCounters()
        _check(self._lib.vc_server_stats(self._h, ctypes.byref(c)), "vc_server_stats")
        return c.as_dict()

    def close(self):
        if self._h:
            _check(self._lib.vc_server_destroy(self._h), "vc_server_destroy")
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchPlan:
    """Batched MVC captured as one CUDA graph (include/vc_plan.h): build once, launch many times.

        plan = BatchPlan(vtx, edge, offsets, neighbors)
        plan.launch(stream); sizes, covers, stats = plan.results(stream)
    """

    def __init__(self, vtx, edge, offsets, neighbors, config: Config | None = None):
        lib = load()
        self._lib = lib
        vtx = _host_i32(vtx)
        edge = _host_i32(edge)
        self.G = vtx.size - 1
        self.total_n = int(vtx[-1])
        on_dev = _is_cuda_tensor(offsets)
        if on_dev:
            off_t, nb_t = _device_csr(offsets, neighbors)  # held until the plan has copied them
            off_p, nb_p = off_t.data_ptr(), nb_t.data_ptr()
        else:
            o = _host_i32(offsets)
            nbr = _host_i32(neighbors)
            if nbr.size == 0:
                nbr = np.zeros(1, dtype=np.int32)
            self._keep = (o, nbr)
            off_p, nb_p = o.ctypes.data, nbr.ctypes.data
        h = ctypes.c_void_p()
        _check(lib.vc_plan_create_mvc_batch(self.G, vtx.ctypes.data, edge.ctypes.data, off_p, nb_p,
                                            1 if on_dev else 0, ctypes.byref(config) if config else None,
                                            ctypes.byref(h)), "vc_plan_create_mvc_batch")
        self._h = h

    def launch(self, stream=None):
        _check(self._lib.vc_plan_launch(self._h, _stream(stream)), "vc_plan_launch")

    def results(self, stream=None, want_covers: bool = False):
        sizes = np.zeros(max(self.G, 1), dtype=np.int32)
        covers = np.zeros(max(self.total_n, 1), dtype=np.int32) if want_covers else None
        st = Stats()
        _check(self._lib.vc_plan_results(self._h, _stream(stream), sizes.ctypes.data,
                                         covers.ctypes.data if covers is not None else None, 0,
                                         ctypes.byref(st)), "vc_plan_results")
        return sizes[: self.G], covers, st.as_dict()

    def completion_ms(self, stream=None) -> np.ndarray:
        """Per graph of the last launch: when it was answered, in ms after the greedy pass's start
        (vc_plan_completion_ns)."""
        out = np.zeros(max(self.G, 1), dtype=np.int64)
        _check(self._lib.vc_plan_completion_ns(self._h, _stream(stream), out.ctypes.data), "vc_plan_completion_ns")
        return out[: self.G].astype(np.float64) * 1e-6

    def close(self):
        if getattr(self, "_h", None):
            _check(self._lib.vc_plan_destroy(self._h), "vc_plan_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
