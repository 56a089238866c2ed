"""Thin ctypes binding of libdgec.so (include/dgec.h).

Argument marshalling only: every step of the computation runs in the CUDA
library. PyTorch supplies device memory (the workspace) and the stream.
There is no CPU path: if the library is missing or no GPU is present the
calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# the in-tree build; DGEC_LIBRARY may name another build of the same library
LIB_PATH = os.environ.get("DGEC_LIBRARY") or os.path.join(_HERE, "_lib", "libdgec.so")

DGEC_OK = 0
STATUS = {0: "DGEC_OK", 1: "DGEC_ERR_INVALID_ARG", 2: "DGEC_ERR_VERTEX_RANGE",
          3: "DGEC_ERR_SELF_LOOP", 4: "DGEC_ERR_TOO_LARGE", 5: "DGEC_ERR_OOM",
          6: "DGEC_ERR_CUDA", 7: "DGEC_ERR_TIMEOUT", 8: "DGEC_ERR_ADMISSION",
          9: "DGEC_ERR_INTERNAL"}

EXPORTS = ["dgec_create", "dgec_destroy", "dgec_last_error", "dgec_status_string",
           "dgec_workspace_size", "dgec_run", "dgec_run_host", "dgec_last_launch_count",
           "dgec_set_kernel_timing", "dgec_kernel_timing", "dgec_stage_timing", "dgec_set_launch_config",
           "dgec_get_launch_config", "dgec_msf_static",
           "dgec_batch_workspace_size", "dgec_run_batch", "dgec_server_create", "dgec_submit",
           "dgec_wait", "dgec_server_lane_capacity", "dgec_server_destroy",
           "dgec_levels_workspace_size", "dgec_run_levels", "dgec_hyper_workspace_size",
           "dgec_run_hyper"]

LEVELS_DENSE = 1
MAX_LEVELS = 64


class LaunchConfig(ctypes.Structure):
    _fields_ = [("knn_block", ctypes.c_int32), ("stream_ctas", ctypes.c_int32),
                ("knn_packed", ctypes.c_int32)]


class DgecError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


CUTOFF = 1
MRD = 2
NEARLY_CAUSAL = 4


class Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("min_cluster_size", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("delta_max", ctypes.c_int64), ("delta_nc", ctypes.c_int64)]


def _params(k, min_cluster_size, delta_max=None, mrd=False, delta_nc=None):
    flags = ((CUTOFF if delta_max is not None else 0) | (MRD if mrd else 0) |
             (NEARLY_CAUSAL if delta_nc is not None else 0))
    return Params(k, min_cluster_size, flags, int(delta_max) if delta_max is not None else 0,
                  int(delta_nc) if delta_nc is not None else 0)


_P = ctypes.c_void_p


class Result(ctypes.Structure):
    _fields_ = [(n, _P) for n in (
        "out_off", "in_off", "out_t", "in_t", "out_id", "in_id", "pos_out", "pos_in", "sk_u", "sk_v", "sk_w",
        "knn_id", "core", "mst_u", "mst_v", "mst_w", "link_a", "link_b", "link_size",
        "fall_cluster", "fall_lambda", "cl_id", "cl_parent", "cl_birth", "cl_death",
        "cl_stab_hi", "cl_stab_lo", "cl_size", "cl_selected", "labels")] + [
        ("n_skeleton", ctypes.c_int64), ("n_mst", ctypes.c_int64),
        ("n_condensed", ctypes.c_int64), ("n_clusters", ctypes.c_int32)]


class BatchResult(ctypes.Structure):
    _fields_ = [(n, _P) for n in (
        "labels", "knn_id", "core", "mst_u", "mst_v", "mst_w", "link_a", "link_b", "link_size",
        "n_clusters", "mst_off", "knn_off")] + [
        ("total_edges", ctypes.c_int64), ("total_mst", ctypes.c_int64),
        ("total_clusters", ctypes.c_int32), ("glob", Result)]


class LevelsParams(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int32), ("h_omega", _P),
                ("min_cluster_size", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class LevelsResult(ctypes.Structure):
    _fields_ = [(n, _P) for n in (
        "sk_u", "sk_v", "sk_w", "merge_level", "merge_parent", "n_components", "level_labels",
        "labels")] + [("n_skeleton", ctypes.c_int64), ("n_merges", ctypes.c_int64),
                      ("n_clusters", ctypes.c_int32)]


class HyperParams(ctypes.Structure):
    _fields_ = [("directed", ctypes.c_int32), ("min_cluster_size", ctypes.c_int32),
                ("flags", ctypes.c_uint32)]


class HyperResult(ctypes.Structure):
    _fields_ = [(n, _P) for n in (
        "src_voff", "src_list", "dst_voff", "dst_list", "sk_u", "sk_v", "sk_w", "mst_u", "mst_v",
        "mst_w", "link_a", "link_b", "link_size", "labels")] + [
        ("n_skeleton", ctypes.c_int64), ("n_mst", ctypes.c_int64), ("n_clusters", ctypes.c_int32)]


class Job(ctypes.Structure):
    _fields_ = [("d_src", _P), ("d_dst", _P), ("d_t", _P), ("n_edges", ctypes.c_int64),
                ("k", ctypes.c_int32), ("min_cluster_size", ctypes.c_int32), ("d_labels", _P)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libdgec.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"dgec CUDA library not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    L.dgec_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int]
    L.dgec_destroy.argtypes = [_P]
    L.dgec_last_error.argtypes = [_P]
    L.dgec_last_error.restype = ctypes.c_char_p
    L.dgec_status_string.argtypes = [ctypes.c_int]
    L.dgec_status_string.restype = ctypes.c_char_p
    L.dgec_workspace_size.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(Params),
                                      ctypes.POINTER(ctypes.c_size_t)]
    L.dgec_run.argtypes = [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int32,
                           ctypes.POINTER(Params), _P, ctypes.c_size_t, _P,
                           ctypes.POINTER(Result)]
    L.dgec_run_host.argtypes = [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int32,
                                ctypes.POINTER(Params), _P, ctypes.c_size_t, _P, _P,
                                ctypes.POINTER(ctypes.c_int32)]
    L.dgec_last_launch_count.argtypes = [_P]
    L.dgec_last_launch_count.restype = ctypes.c_int64
    L.dgec_set_kernel_timing.argtypes = [_P, ctypes.c_int, ctypes.c_char_p]
    L.dgec_kernel_timing.argtypes = [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                     ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_int64)]
    L.dgec_stage_timing.argtypes = [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                    ctypes.POINTER(ctypes.c_double)]
    L.dgec_set_launch_config.argtypes = [_P, ctypes.POINTER(LaunchConfig)]
    L.dgec_get_launch_config.argtypes = [_P, ctypes.POINTER(LaunchConfig)]
    I64A = ctypes.POINTER(ctypes.c_int64)
    I32A = ctypes.POINTER(ctypes.c_int32)
    L.dgec_batch_workspace_size.argtypes = [ctypes.c_int32, I64A, I32A, I32A, I32A,
                                            ctypes.POINTER(ctypes.c_size_t)]
    L.dgec_run_batch.argtypes = [_P, ctypes.c_int32, I64A, I32A, I32A, I32A, _P, _P, _P, _P,
                                 ctypes.c_size_t, _P, ctypes.POINTER(BatchResult)]
    L.dgec_server_create.argtypes = [ctypes.c_int, _P, ctypes.c_size_t, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_P)]
    L.dgec_submit.argtypes = [_P, ctypes.POINTER(Job), ctypes.POINTER(ctypes.c_uint64)]
    L.dgec_wait.argtypes = [_P, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                            ctypes.POINTER(ctypes.c_double)]
    L.dgec_server_lane_capacity.argtypes = [_P]
    L.dgec_server_lane_capacity.restype = ctypes.c_int64
    L.dgec_server_destroy.argtypes = [_P]
    L.dgec_levels_workspace_size.argtypes = [ctypes.c_int64, ctypes.c_int32,
                                             ctypes.POINTER(LevelsParams),
                                             ctypes.POINTER(ctypes.c_size_t)]
    L.dgec_run_levels.argtypes = [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int32,
                                  ctypes.POINTER(LevelsParams), _P, ctypes.c_size_t, _P,
                                  ctypes.POINTER(LevelsResult)]
    L.dgec_hyper_workspace_size.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                            ctypes.c_int64, ctypes.POINTER(HyperParams),
                                            ctypes.POINTER(ctypes.c_size_t)]
    L.dgec_run_hyper.argtypes = [_P, _P, ctypes.c_int64, ctypes.c_int32, _P, _P, ctypes.c_int64, _P, _P,
                                 ctypes.c_int64, ctypes.POINTER(HyperParams), _P, ctypes.c_size_t, _P,
                                 ctypes.POINTER(HyperResult)]
    L.dgec_msf_static.argtypes = [_P, _P, _P, ctypes.c_int64, ctypes.c_int64, _P, _P, _P,
                                  ctypes.POINTER(ctypes.c_int64), _P]
    _lib = L
    return L


def msf_static(u, v, w, n_nodes: int, out_u, out_v, out_w, stream=None) -> int:
    """Minimum spanning forest through the allocation-free entry point: the
    caller's device tensors in (u < v, int32; w >= 0, int64; all of one
    length) and out (int32, int32, int64, each with room for n_nodes - 1
    edges), all on one device; the library uses only its fixed internal
    array. Runs on `stream` (default: that device's current stream).
    Returns the number of forest edges written."""
    import torch
    L = load()
    if not hasattr(u, "is_cuda") or not u.is_cuda:
        raise ValueError("u must be a CUDA tensor")
    dev = u.device.index
    n = int(u.shape[0]) if u.dim() == 1 else -1
    _dev("u", u, torch.int32, n, dev)
    _dev("v", v, torch.int32, n, dev)
    _dev("w", w, torch.int64, n, dev)
    need = max(int(n_nodes) - 1, 0)
    for name, x, dt in (("out_u", out_u, torch.int32), ("out_v", out_v, torch.int32),
                        ("out_w", out_w, torch.int64)):
        _dev(name, x, dt, None, dev)
        if int(x.shape[0]) < need:
            raise ValueError(f"{name} has {int(x.shape[0])} elements, needs at least {need}")
    with torch.cuda.device(dev):
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        m = ctypes.c_int64(0)
        rc = L.dgec_msf_static(u.data_ptr(), v.data_ptr(), w.data_ptr(), n, int(n_nodes),
                               out_u.data_ptr(), out_v.data_ptr(), out_w.data_ptr(), ctypes.byref(m),
                               st.cuda_stream)
    if rc != DGEC_OK:
        raise DgecError(rc, L.dgec_status_string(rc).decode())
    return int(m.value)


def workspace_size(n_edges: int, n_vertices: int, k: int, min_cluster_size: int, mrd: bool = False,
                   delta_nc=None) -> int:
    L = load()
    p = _params(k, min_cluster_size, None, mrd, delta_nc)
    out = ctypes.c_size_t(0)
    rc = L.dgec_workspace_size(n_edges, n_vertices, ctypes.byref(p), ctypes.byref(out))
    if rc != DGEC_OK:
        raise DgecError(rc, L.dgec_status_string(rc).decode())
    return int(out.value)


def _dev(name, x, dtype, n, device):
    """A device argument must be a contiguous 1-D tensor of `dtype` with `n`
    elements on cuda:`device`: the kernels read exactly that many."""
    if (not hasattr(x, "is_cuda") or x.dtype != dtype or not x.is_cuda or not x.is_contiguous()
            or x.dim() != 1 or x.device.index != device):
        raise ValueError(f"{name} must be a contiguous 1-D {dtype} tensor on cuda:{device}")
    if n is not None and int(x.shape[0]) != n:
        raise ValueError(f"{name} has {int(x.shape[0])} elements, expected {n}")


def _host(name, a, dtype, n, writeable=False):
    """A host argument must be a C-contiguous 1-D numpy array of `dtype` with
    `n` elements: the library copies exactly that many bytes from (or to) it."""
    if (not isinstance(a, np.ndarray) or a.dtype != dtype or a.ndim != 1 or not a.flags.c_contiguous
            or (writeable and not a.flags.writeable)):
        raise ValueError(f"{name} must be a {'writeable ' if writeable else ''}C-contiguous 1-D numpy "
                         f"{np.dtype(dtype).name} array")
    if a.shape[0] != n:
        raise ValueError(f"{name} has {a.shape[0]} elements, expected {n}")


class Context:
    """A dgec context on one CUDA device plus a reusable torch workspace."""

    def __init__(self, device: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("dgec needs a CUDA device; there is no CPU path")
        self.torch = torch
        self.L = load()
        self.device = device
        h = _P()
        rc = self.L.dgec_create(ctypes.byref(h), device)
        if rc != DGEC_OK:
            raise DgecError(rc, "dgec_create failed")
        self.h = h
        self.ws = None

    def close(self):
        if self.h:
            self.L.dgec_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != DGEC_OK:
            raise DgecError(rc, self.L.dgec_last_error(self.h).decode())

    def workspace(self, nbytes: int):
        torch = self.torch
        if self.ws is None or self.ws.numel() < nbytes:
            self.ws = None
            self.ws = torch.empty(nbytes, dtype=torch.uint8, device=f"cuda:{self.device}")
        return self.ws

    def _stream(self, stream, ws):
        """The launch stream: the current one by default. A workspace used on
        another stream is recorded there, so that the caching allocator does
        not hand its memory out again while that stream still uses it."""
        cur = self.torch.cuda.current_stream(self.device)
        if stream is None:
            return cur
        if stream != cur:
            ws.record_stream(stream)
        return stream

    def _graph_args(self, src, dst, t):
        torch = self.torch
        E = int(src.shape[0]) if hasattr(src, "shape") and len(src.shape) == 1 else -1
        _dev("src", src, torch.int32, None, self.device)
        _dev("dst", dst, torch.int32, E, self.device)
        _dev("t", t, torch.int64, E, self.device)
        return E

    def launches(self) -> int:
        return int(self.L.dgec_last_launch_count(self.h))

    def set_kernel_timing(self, mode: int, name: str | None = None):
        """0 off, 1 only kernel `name`, 2 every launch, 3 kernels whose name
        starts with `name` (resets totals)."""
        self._check(self.L.dgec_set_kernel_timing(self.h, mode, name.encode() if name else None))

    def kernel_timing(self) -> dict:
        """{kernel name: (total ms, launches)} since the last reset."""
        out = {}
        i = 0
        while True:
            nm = ctypes.c_char_p()
            ms = ctypes.c_double()
            n = ctypes.c_int64()
            rc = self.L.dgec_kernel_timing(self.h, i, ctypes.byref(nm), ctypes.byref(ms),
                                           ctypes.byref(n))
            if rc != DGEC_OK:
                break
            out[nm.value.decode()] = (ms.value, n.value)
            i += 1
        return out

    def set_launch_config(self, knn_block: int, stream_ctas: int, knn_packed: int = 2):
        """Threads per CTA of the kNN kernel, CTAs of the grid-stride
        streaming kernels and the kNN form (0 separate time and id arrays,
        1 packed 64-bit keys one edge a thread, 2 packed keys in list order)
        for the calls on this context (speed only)."""
        cfg = LaunchConfig(knn_block, stream_ctas, knn_packed)
        self._check(self.L.dgec_set_launch_config(self.h, ctypes.byref(cfg)))

    def launch_config(self) -> tuple:
        c = LaunchConfig()
        self._check(self.L.dgec_get_launch_config(self.h, ctypes.byref(c)))
        return int(c.knn_block), int(c.stream_ctas), int(c.knn_packed)

    def stage_timing(self) -> list:
        """[(stage name, device ms)] of the last completed call, in order."""
        out = []
        i = 0
        while True:
            nm = ctypes.c_char_p()
            ms = ctypes.c_double()
            if self.L.dgec_stage_timing(self.h, i, ctypes.byref(nm), ctypes.byref(ms)) != DGEC_OK:
                break
            out.append((nm.value.decode(), ms.value))
            i += 1
        return out

    def run(self, src, dst, t, n_vertices: int, k: int, min_cluster_size: int, stream=None,
            delta_max=None, mrd: bool = False, delta_nc=None):
        """Alg. 4 on device tensors (int32 src/dst, int64 t). Returns an
        Output whose tensors view the workspace (valid until the next run).
        delta_max: the time cutoff of Sec. 4.3 (None = no cutoff); mrd: cluster
        the mutual-reachability graph (an approximation, see dgec.h);
        delta_nc: the nearly-causal tolerance of Sec. 4.3 (None = causal)."""
        E = self._graph_args(src, dst, t)
        p = _params(k, min_cluster_size, delta_max, mrd, delta_nc)
        need = workspace_size(E, n_vertices, k, min_cluster_size, mrd, delta_nc)
        ws = self.workspace(need)
        st = self._stream(stream, ws)
        res = Result()
        rc = self.L.dgec_run(self.h, src.data_ptr(), dst.data_ptr(), t.data_ptr(), E, n_vertices,
                             ctypes.byref(p), ws.data_ptr(), ws.numel(), st.cuda_stream,
                             ctypes.byref(res))
        self._check(rc)
        return Output(res, ws, E, n_vertices, k)

    def run_levels(self, src, dst, t, n_vertices: int, omega, min_cluster_size: int = 0,
                   dense: bool = False, stream=None):
        """Discrete dendrogram (Alg. 5) at thresholds `omega` on device tensors,
        plus condensed labels when min_cluster_size >= 2. Returns a
        LevelsOutput viewing the workspace (valid until the next run)."""
        E = self._graph_args(src, dst, t)
        om = np.ascontiguousarray(omega, dtype=np.int64)
        p = LevelsParams(len(om), om.ctypes.data, min_cluster_size, LEVELS_DENSE if dense else 0)
        nb = ctypes.c_size_t(0)
        self._check(self.L.dgec_levels_workspace_size(E, n_vertices, ctypes.byref(p), ctypes.byref(nb)))
        ws = self.workspace(nb.value)
        st = self._stream(stream, ws)
        res = LevelsResult()
        rc = self.L.dgec_run_levels(self.h, src.data_ptr(), dst.data_ptr(), t.data_ptr(), E,
                                    n_vertices, ctypes.byref(p), ws.data_ptr(), ws.numel(),
                                    st.cuda_stream, ctypes.byref(res))
        self._check(rc)
        return LevelsOutput(res, ws, E, len(om))

    def run_hyper(self, t, s_off, s_vert, n_vertices: int, min_cluster_size: int, d_off=None,
                  d_vert=None, stream=None):
        """Alg. 1 on a dynamic hypergraph (Sec. 4.4) given as device tensors:
        t int64[E], member rows s_off int64[E+1] / s_vert int32[Ms], and for a
        directed hypergraph target rows d_off / d_vert (sources in s_*)."""
        torch = self.torch
        directed = d_off is not None
        if directed != (d_vert is not None):
            raise ValueError("a directed hypergraph needs both d_off and d_vert")
        _dev("t", t, torch.int64, None, self.device)
        E = int(t.shape[0])
        _dev("s_off", s_off, torch.int64, E + 1, self.device)
        _dev("s_vert", s_vert, torch.int32, None, self.device)
        Ms = int(s_vert.shape[0])
        Md = 0
        if directed:
            _dev("d_off", d_off, torch.int64, E + 1, self.device)
            _dev("d_vert", d_vert, torch.int32, None, self.device)
            Md = int(d_vert.shape[0])
        p = HyperParams(1 if directed else 0, min_cluster_size, 0)
        nb = ctypes.c_size_t(0)
        self._check(self.L.dgec_hyper_workspace_size(E, n_vertices, Ms, Md, ctypes.byref(p), ctypes.byref(nb)))
        ws = self.workspace(nb.value)
        st = self._stream(stream, ws)
        res = HyperResult()
        rc = self.L.dgec_run_hyper(self.h, t.data_ptr(), E, n_vertices, s_off.data_ptr(), s_vert.data_ptr(), Ms,
                                   d_off.data_ptr() if directed else None,
                                   d_vert.data_ptr() if directed else None, Md, ctypes.byref(p),
                                   ws.data_ptr(), ws.numel(), st.cuda_stream, ctypes.byref(res))
        self._check(rc)
        return HyperOutput(res, ws, E, n_vertices, Ms, Md)

    def run_batch(self, src, dst, t, edge_off, n_vertices, k, min_cluster_size, stream=None):
        """Batched Alg. 4 over graphs laid end to end on the device; tables are
        host arrays (edge_off[G+1] starting at 0, n_vertices/k/M per graph)."""
        return _run_batch(self, src, dst, t, edge_off, n_vertices, k, min_cluster_size, stream)

    def run_batch_passes(self, src, dst, t, edge_off, n_vertices, k, min_cluster_size, max_edges: int,
                         labels_out, stream=None):
        """Every graph of a batch too large for one workspace, in passes of
        consecutive graphs holding at most max_edges edges (a larger graph
        gets a pass of its own). Graph g's labels land in labels_out (device
        int32[total]) at edge_off[g], exactly as dgec_run_batch (or dgec_run)
        gives them for that graph alone. Returns (n_clusters per graph as a
        host array, number of passes)."""
        torch = self.torch
        eo = np.ascontiguousarray(edge_off, np.int64)
        G = len(eo) - 1
        total = int(eo[-1]) if G >= 0 else 0
        _dev("labels_out", labels_out, torch.int32, total, self.device)
        nv = np.ascontiguousarray(n_vertices, np.int32)
        kk = np.ascontiguousarray(k, np.int32)
        mm = np.ascontiguousarray(min_cluster_size, np.int32)
        ncl = np.zeros(max(G, 0), np.int32)
        passes = 0
        g0 = 0
        while g0 < G:
            g1 = int(np.searchsorted(eo, eo[g0] + int(max_edges), side="right")) - 1
            g1 = min(max(g1, g0 + 1), G)
            a, b = int(eo[g0]), int(eo[g1])
            out = _run_batch(self, src[a:b], dst[a:b], t[a:b], eo[g0:g1 + 1] - a, nv[g0:g1], kk[g0:g1],
                             mm[g0:g1], stream)
            st = self._stream(stream, out.t["labels"])
            with torch.cuda.stream(st):
                labels_out[a:b].copy_(out.t["labels"])
                ncl[g0:g1] = out.t["n_clusters"].cpu().numpy()
            passes += 1
            g0 = g1
        return ncl, passes

    def run_host(self, src: np.ndarray, dst: np.ndarray, t: np.ndarray, n_vertices: int, k: int,
                 min_cluster_size: int, labels_out: np.ndarray | None = None, stream=None,
                 delta_max=None, mrd: bool = False, delta_nc=None):
        """Alg. 4 from host arrays (pinned numpy views avoid staging copies);
        returns (labels, n_clusters)."""
        _host("src", src, np.int32, src.shape[0] if isinstance(src, np.ndarray) and src.ndim == 1 else -1)
        E = int(src.shape[0])
        _host("dst", dst, np.int32, E)
        _host("t", t, np.int64, E)
        if labels_out is None:
            labels_out = np.empty(E, np.int32)
        _host("labels_out", labels_out, np.int32, E, writeable=True)
        p = _params(k, min_cluster_size, delta_max, mrd, delta_nc)
        need = workspace_size(E, n_vertices, k, min_cluster_size, mrd, delta_nc) + 16 * E + 4096
        ws = self.workspace(need)
        st = self._stream(stream, ws)
        ncl = ctypes.c_int32(0)
        rc = self.L.dgec_run_host(self.h, src.ctypes.data, dst.ctypes.data, t.ctypes.data, E,
                                  n_vertices, ctypes.byref(p), ws.data_ptr(), ws.numel(),
                                  st.cuda_stream, labels_out.ctypes.data, ctypes.byref(ncl))
        self._check(rc)
        return labels_out, int(ncl.value)


def _i64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _i32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def batch_workspace_size(edge_off, n_vertices, k, min_cluster_size) -> int:
    L = load()
    eo = np.ascontiguousarray(edge_off, np.int64)
    nv = np.ascontiguousarray(n_vertices, np.int32)
    kk = np.ascontiguousarray(k, np.int32)
    mm = np.ascontiguousarray(min_cluster_size, np.int32)
    out = ctypes.c_size_t(0)
    rc = L.dgec_batch_workspace_size(len(nv), _i64p(eo), _i32p(nv), _i32p(kk), _i32p(mm),
                                     ctypes.byref(out))
    if rc != DGEC_OK:
        raise DgecError(rc, L.dgec_status_string(rc).decode())
    return int(out.value)


def _run_batch(ctx, src, dst, t, edge_off, n_vertices, k, min_cluster_size, stream=None):
    torch = ctx.torch
    eo = np.ascontiguousarray(edge_off, np.int64)
    nv = np.ascontiguousarray(n_vertices, np.int32)
    kk = np.ascontiguousarray(k, np.int32)
    mm = np.ascontiguousarray(min_cluster_size, np.int32)
    G = len(nv)
    n = int(eo[-1]) if len(eo) else 0
    _dev("src", src, torch.int32, n, ctx.device)
    _dev("dst", dst, torch.int32, n, ctx.device)
    _dev("t", t, torch.int64, n, ctx.device)
    need = batch_workspace_size(eo, nv, kk, mm)
    ws = ctx.workspace(need)
    st = ctx._stream(stream, ws)
    res = BatchResult()
    rc = ctx.L.dgec_run_batch(ctx.h, G, _i64p(eo), _i32p(nv), _i32p(kk), _i32p(mm),
                              src.data_ptr(), dst.data_ptr(), t.data_ptr(), ws.data_ptr(),
                              ws.numel(), st.cuda_stream, ctypes.byref(res))
    ctx._check(rc)
    return BatchOutput(res, ws, eo, kk)


class BatchOutput:
    """Per-graph results of a batch (device views of the workspace)."""

    def __init__(self, res, ws, edge_off, k):
        import torch
        self.G = len(k)
        self.edge_off = edge_off
        self.k = k
        E = int(res.total_edges)
        nmst = int(res.total_mst)
        base = ws.data_ptr()

        def view(ptr, n, dt, sz):
            if n == 0 or ptr is None:
                return torch.empty(0, dtype=dt, device=ws.device)
            off = ptr - base
            return ws[off:off + n * sz].view(dt)
        knn_total = int(np.sum((edge_off[1:] - edge_off[:-1]) * k))
        self.t = {
            "labels": view(res.labels, E, torch.int32, 4),
            "knn_id": view(res.knn_id, knn_total, torch.int32, 4),
            "core": view(res.core, E, torch.int64, 8),
            "mst_u": view(res.mst_u, nmst, torch.int32, 4),
            "mst_v": view(res.mst_v, nmst, torch.int32, 4),
            "mst_w": view(res.mst_w, nmst, torch.int64, 8),
            "link_a": view(res.link_a, nmst, torch.int32, 4),
            "link_b": view(res.link_b, nmst, torch.int32, 4),
            "link_size": view(res.link_size, nmst, torch.int64, 8),
            "n_clusters": view(res.n_clusters, self.G, torch.int32, 4),
            "mst_off": view(res.mst_off, self.G + 1, torch.int64, 8),
            "knn_off": view(res.knn_off, self.G + 1, torch.int64, 8),
        }
        self.total_clusters = int(res.total_clusters)

    def numpy(self, name):
        return self.t[name].cpu().numpy()

    def graph(self, g):
        """Host copies of graph g's outputs (local ids)."""
        eo = self.edge_off
        a, b = int(eo[g]), int(eo[g + 1])
        mo = self.numpy("mst_off")
        ko = self.numpy("knn_off")
        m0, m1 = int(mo[g]), int(mo[g + 1])
        kk = int(self.k[g])
        out = {
            "labels": self.t["labels"][a:b].cpu().numpy(),
            "core": self.t["core"][a:b].cpu().numpy(),
            "knn_id": self.t["knn_id"][int(ko[g]):int(ko[g + 1])].cpu().numpy().reshape(b - a, kk),
            "n_clusters": int(self.numpy("n_clusters")[g]),
        }
        for n in ("mst_u", "mst_v", "mst_w", "link_a", "link_b", "link_size"):
            out[n] = self.t[n][m0:m1].cpu().numpy()
        return out


class Server:
    """Serving loop (continuous batching) over a torch-allocated device pool.
    Jobs are device tensors (views of a resident stream are fine); submit()
    returns at once, wait() gives (status, n_clusters, latency_ms)."""

    def __init__(self, pool_bytes: int, n_lanes: int, vertex_bound: int, max_jobs_per_batch: int = 64,
                 device: int = 0):
        import torch
        self.L = load()
        self.pool = torch.empty(pool_bytes, dtype=torch.uint8, device=f"cuda:{device}")
        h = _P()
        rc = self.L.dgec_server_create(device, self.pool.data_ptr(), pool_bytes, n_lanes,
                                       vertex_bound, max_jobs_per_batch, ctypes.byref(h))
        if rc != DGEC_OK:
            raise DgecError(rc, "dgec_server_create failed")
        self.h = h
        self.device = device
        self._keep = {}

    def lane_capacity(self) -> int:
        return int(self.L.dgec_server_lane_capacity(self.h))

    def submit(self, src, dst, t, k: int, min_cluster_size: int, labels) -> int:
        import torch
        E = int(src.shape[0]) if hasattr(src, "shape") and len(src.shape) == 1 else -1
        _dev("src", src, torch.int32, None, self.device)
        _dev("dst", dst, torch.int32, E, self.device)
        _dev("t", t, torch.int64, E, self.device)
        _dev("labels", labels, torch.int32, E, self.device)
        j = Job(src.data_ptr(), dst.data_ptr(), t.data_ptr(), int(src.shape[0]), k,
                min_cluster_size, labels.data_ptr())
        tk = ctypes.c_uint64(0)
        rc = self.L.dgec_submit(self.h, ctypes.byref(j), ctypes.byref(tk))
        if rc != DGEC_OK:
            raise DgecError(rc, "dgec_submit failed")
        self._keep[tk.value] = (src, dst, t, labels)  # keep the tensors alive
        return int(tk.value)

    def wait(self, ticket: int, timeout_ms: int = -1):
        n = ctypes.c_int32(0)
        lat = ctypes.c_double(0)
        rc = self.L.dgec_wait(self.h, ticket, timeout_ms, ctypes.byref(n), ctypes.byref(lat))
        if rc != 7:  # a timed-out job is still pending
            self._keep.pop(ticket, None)
        return rc, int(n.value), float(lat.value)

    def close(self):
        if self.h:
            self.L.dgec_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Output:
    """Device-resident results of one run, as torch views of the workspace."""

    _SPEC = {  # name -> (dtype, length expression)
        "out_off": ("int64", "V+1"), "in_off": ("int64", "V+1"),
        "out_t": ("int64", "E"), "in_t": ("int64", "E"),
        "out_id": ("int32", "E"), "in_id": ("int32", "E"),
        "pos_out": ("int32", "E"), "pos_in": ("int32", "E"),
        "sk_u": ("int32", "nsk"), "sk_v": ("int32", "nsk"), "sk_w": ("int64", "nsk"),
        "knn_id": ("int32", "E*k"), "core": ("int64", "E"),
        "mst_u": ("int32", "nmst"), "mst_v": ("int32", "nmst"), "mst_w": ("int64", "nmst"),
        "link_a": ("int32", "nmst"), "link_b": ("int32", "nmst"), "link_size": ("int64", "nmst"),
        "fall_cluster": ("int32", "E"), "fall_lambda": ("uint64", "E"),
        "cl_id": ("int32", "ncl"), "cl_parent": ("int32", "ncl"),
        "cl_birth": ("uint64", "ncl"), "cl_death": ("uint64", "ncl"),
        "cl_stab_hi": ("uint64", "ncl"), "cl_stab_lo": ("uint64", "ncl"),
        "cl_size": ("int64", "ncl"), "cl_selected": ("int32", "ncl"),
        "labels": ("int32", "E"),
    }

    def __init__(self, res: Result, ws, E, V, k):
        import torch
        self.n_skeleton = int(res.n_skeleton)
        self.n_mst = int(res.n_mst)
        self.n_condensed = int(res.n_condensed)
        self.n_clusters = int(res.n_clusters)
        env = dict(E=E, V=V, k=k, nsk=self.n_skeleton, nmst=self.n_mst, ncl=self.n_condensed)
        base = ws.data_ptr()
        dts = {"int32": (torch.int32, 4), "int64": (torch.int64, 8), "uint64": (torch.int64, 8)}
        self._raw = {}
        for name, (dt, expr) in self._SPEC.items():
            ptr = getattr(res, name)
            n = int(eval(expr, {}, env))
            tdt, sz = dts[dt]
            if n == 0 or ptr is None:
                self._raw[name] = (torch.empty(0, dtype=tdt, device=ws.device), dt)
                continue
            off = ptr - base
            self._raw[name] = (ws[off:off + n * sz].view(tdt), dt)
        self.E, self.V, self.k = E, V, k

    def tensor(self, name):
        return self._raw[name][0]

    def numpy(self, name):
        t, dt = self._raw[name]
        a = t.cpu().numpy()
        if dt == "uint64":
            a = a.view(np.uint64)
        if name == "knn_id":
            a = a.reshape(self.E, self.k)
        return a


class LevelsOutput:
    """Device-resident results of one discrete-dendrogram run."""

    def __init__(self, res: LevelsResult, ws, E, q):
        import torch
        self.n_skeleton = int(res.n_skeleton)
        self.n_merges = int(res.n_merges)
        self.n_clusters = int(res.n_clusters)
        self.E, self.q = E, q
        spec = {"sk_u": (torch.int32, 4, self.n_skeleton), "sk_v": (torch.int32, 4, self.n_skeleton),
                "sk_w": (torch.int64, 8, self.n_skeleton), "merge_level": (torch.int32, 4, E),
                "merge_parent": (torch.int32, 4, E), "n_components": (torch.int64, 8, q),
                "level_labels": (torch.int32, 4, q * E), "labels": (torch.int32, 4, E)}
        base = ws.data_ptr()
        self._t = {}
        for name, (dt, sz, n) in spec.items():
            ptr = getattr(res, name)
            if ptr is None or n == 0:
                self._t[name] = None if ptr is None else torch.empty(0, dtype=dt, device=ws.device)
                continue
            off = ptr - base
            self._t[name] = ws[off:off + n * sz].view(dt)

    def tensor(self, name):
        return self._t[name]

    def numpy(self, name):
        t = self._t[name]
        if t is None:
            return None
        a = t.cpu().numpy()
        if name == "level_labels":
            a = a.reshape(self.q, self.E)
        return a


class HyperOutput:
    """Device-resident results of one hypergraph run."""

    def __init__(self, res: HyperResult, ws, E, V, Ms, Md):
        import torch
        self.n_skeleton = int(res.n_skeleton)
        self.n_mst = int(res.n_mst)
        self.n_clusters = int(res.n_clusters)
        i32, i64 = (torch.int32, 4), (torch.int64, 8)
        spec = {"src_voff": (i64, V + 1), "src_list": (i32, Ms), "dst_voff": (i64, V + 1),
                "dst_list": (i32, Md), "sk_u": (i32, self.n_skeleton), "sk_v": (i32, self.n_skeleton),
                "sk_w": (i64, self.n_skeleton), "mst_u": (i32, self.n_mst), "mst_v": (i32, self.n_mst),
                "mst_w": (i64, self.n_mst), "link_a": (i32, self.n_mst), "link_b": (i32, self.n_mst),
                "link_size": (i64, self.n_mst), "labels": (i32, E)}
        base = ws.data_ptr()
        self._t = {}
        for name, ((dt, sz), n) in spec.items():
            ptr = getattr(res, name)
            if ptr is None:
                self._t[name] = None
            elif n == 0:
                self._t[name] = torch.empty(0, dtype=dt, device=ws.device)
            else:
                self._t[name] = ws[ptr - base:ptr - base + n * sz].view(dt)

    def tensor(self, name):
        return self._t[name]

    def numpy(self, name):
        t = self._t[name]
        return None if t is None else t.cpu().numpy()
