"""ctypes binding of libakmc (include/akmc.h): argument marshalling only.

PyTorch provides the device workspace and the stream; every step of the
AKMC path runs in the library's CUDA kernels.  There is no fallback: if the
compiled library or a CUDA device is missing, the constructor raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libakmc.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ETRAPPED, ENUMERIC = range(7)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ETRAPPED", 6: "ENUMERIC"}

_lock = threading.Lock()
_lib = None


class AkmcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class VoxelDescC(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("n_vac", ctypes.c_int32), ("frac", ctypes.c_double * 3),
                ("T", ctypes.c_double), ("model", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("uid", ctypes.c_uint64)]


class ModelC(ctypes.Structure):
    _fields_ = [("eps1", ctypes.c_double * 25), ("eps2", ctypes.c_double * 25),
                ("E0", ctypes.c_double * 4), ("nu", ctypes.c_double), ("a", ctypes.c_double),
                ("r_cut", ctypes.c_double), ("n_r", ctypes.c_int32), ("n_rho", ctypes.c_int32),
                ("rho_h", ctypes.c_double), ("phi_tab", ctypes.c_void_p), ("f_tab", ctypes.c_void_p),
                ("F_tab", ctypes.c_void_p)]


class StateC(ctypes.Structure):
    _fields_ = [("species", ctypes.c_void_p), ("vac_pos", ctypes.c_void_p), ("vac_disp", ctypes.c_void_p),
                ("rates", ctypes.c_void_p), ("dE", ctypes.c_void_p), ("event_log", ctypes.c_void_p),
                ("t_hi", ctypes.c_double), ("t_lo", ctypes.c_double), ("n_events", ctypes.c_uint64),
                ("status", ctypes.c_int32), ("L", ctypes.c_int32), ("n_vac", ctypes.c_int32)]


def load_library():
    """Load libakmc.so (built by __graft_entry__.build()); raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libakmc.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P, I32, U64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_size_t
        sig = {
            "akmc_workspace_bytes": (SZ, [P, I32, P, I32]),
            "akmc_create_batch": (I32, [P, I32, P, I32, P, SZ, P, ctypes.POINTER(P)]),
            "akmc_compute_rates": (I32, [P, P]),
            "akmc_set_targets": (I32, [P, P, P]),
            "akmc_launch_step": (I32, [P, P]),
            "akmc_reset_voxels": (I32, [P, P, P, I32, P]),
            "akmc_step_n": (I32, [P, P, P]),
            "akmc_step_sublattice": (I32, [P, I32, U64, ctypes.c_uint32, I32, ctypes.c_double, P]),
            "akmc_step_sublattice_async": (I32, [P, I32, U64, ctypes.c_uint32, I32, ctypes.c_double, P]),
            "akmc_test_sublattice_stall": (I32, [P, I32, ctypes.c_uint32, I32, ctypes.c_double, I32, P]),
            "akmc_read_state": (I32, [P, I32, ctypes.POINTER(StateC), P]),
            "akmc_load_state": (I32, [P, I32, P, P, ctypes.c_double, ctypes.c_double, U64, P]),
            "akmc_sync_status": (I32, [P, P, P]),
            "akmc_load_batch_state": (I32, [P, P, P, P, P, P, P]),
            "akmc_read_batch_state": (I32, [P, P, P, P, P, P, P, P, P]),
            "akmc_batch_sites": (SZ, [P]),
            "akmc_batch_vacancies": (ctypes.c_int64, [P]),
            "akmc_cluster_hist": (I32, [P, I32, I32, P, P]),
            "akmc_read_density": (I32, [P, I32, P, P]),
            "akmc_select_scratch_bytes": (SZ, [P, I32]),
            "akmc_select_plan": (I32, [P, I32, P, SZ, P, P]),
            "akmc_select_logits": (I32, [P, P, I32, I32, ctypes.c_float, U64, U64, P, P, P, P]),
            "akmc_cluster_hist_noalloc": (I32, [P, I32, I32, P, P]),
            "akmc_workload_proxy": (I32, [P, P, P, P, P]),
            "akmc_set_launch": (I32, [P, I32, I32]),
            "akmc_n_voxels": (I32, [P]),
            "akmc_destroy_batch": (None, [P]),
            "akmc_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def last_error() -> str:
    return load_library().akmc_last_error().decode()


def _check(st):
    if st != OK:
        raise AkmcError(st, last_error())


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def make_descs(descs) -> ctypes.Array:
    arr = (VoxelDescC * len(descs))()
    for i, d in enumerate(descs):
        c = arr[i]
        c.L, c.n_vac = int(d.L), int(d.n_vac)
        fr = list(d.frac) + [0.0] * (3 - len(d.frac))
        c.frac[:] = [float(x) for x in fr[:3]]
        c.T, c.model, c.precision = float(d.T), int(d.model), int(d.precision)
        c.seed, c.uid = int(d.seed), int(d.uid)
    return arr


class ModelHolder:
    """C view of a model object (eps1, eps2, E0, nu, a, r_cut, rho_h and the
    optional phi_tab/f_tab/F_tab arrays); keeps the arrays alive."""

    def __init__(self, model):
        m = ModelC()
        m.eps1[:] = [float(x) for x in np.asarray(model.eps1, np.float64).ravel()]
        m.eps2[:] = [float(x) for x in np.asarray(model.eps2, np.float64).ravel()]
        m.E0[:] = [float(x) for x in model.E0]
        m.nu, m.a, m.r_cut, m.rho_h = float(model.nu), float(model.a), float(model.r_cut), float(model.rho_h)
        self.keep = []
        if getattr(model, "phi_tab", None) is not None:
            for name in ("phi_tab", "f_tab", "F_tab"):
                arr = np.ascontiguousarray(getattr(model, name), dtype=np.float64)
                self.keep.append(arr)
                setattr(m, name, arr.ctypes.data)
            m.n_r = int(model.phi_tab.shape[1])
            m.n_rho = int(model.F_tab.shape[1])
        self.c = m


def workspace_bytes(descs, model, event_log_capacity=0) -> int:
    lib = load_library()
    cd = make_descs(descs)
    mh = ModelHolder(model)
    n = lib.akmc_workspace_bytes(ctypes.cast(cd, ctypes.c_void_p), len(descs), ctypes.byref(mh.c),
                                 int(event_log_capacity))
    if n == 0:
        raise AkmcError(EINVAL, last_error())
    return int(n)


def cluster_hist_noalloc(species, L, mode, hist, stream=None):
    """Allocation-free Cu cluster histogram of one lattice held by the caller:
    `species` a CUDA uint8 tensor of 2L^3 codes, `hist` a CUDA int64 tensor of
    8 bins that receives the counts (stream-ordered)."""
    import torch
    L = int(L)
    if not (isinstance(species, torch.Tensor) and isinstance(hist, torch.Tensor)):
        raise TypeError("species and hist must be torch tensors")
    if not (species.is_cuda and species.dtype == torch.uint8 and species.is_contiguous()):
        raise ValueError("species must be a contiguous CUDA uint8 tensor")
    if not (hist.is_cuda and hist.dtype == torch.int64 and hist.is_contiguous() and hist.numel() >= 8):
        raise ValueError("hist must be a contiguous CUDA int64 tensor of at least 8 elements")
    if L >= 1 and species.numel() < 2 * L ** 3:
        # the C entry point cannot see the buffer's size: a short buffer would be read past its end
        raise ValueError("species holds %d codes, fewer than 2L^3 = %d" % (species.numel(), 2 * L ** 3))
    if species.device != hist.device:
        raise ValueError("species and hist are on different devices")
    # the static scratch used is that of the current device: run on the tensors' device
    with torch.cuda.device(species.device):
        _check(load_library().akmc_cluster_hist_noalloc(ctypes.c_void_p(species.data_ptr()), L, int(mode),
                                                        ctypes.c_void_p(hist.data_ptr()), _stream_ptr(stream)))


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Batch:
    """A batch of independent voxels resident in one device workspace."""

    def __init__(self, descs: Sequence, model, event_log_capacity: int = 0, device=None, stream=None,
                 workspace=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("akmc needs a CUDA device; there is no CPU fallback")
        self._lib = load_library()
        self.descs = list(descs)
        self.n = len(self.descs)
        self.log_cap = int(event_log_capacity)
        self._cdescs = make_descs(self.descs)
        self._mh = ModelHolder(model)
        self.nbytes = workspace_bytes(self.descs, model, self.log_cap)
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if workspace is None:
            workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=dev)
        if workspace.numel() < self.nbytes:
            raise AkmcError(ENOMEM, "workspace too small")
        self.workspace = workspace
        self.device = dev
        h = ctypes.c_void_p()
        _check(self._lib.akmc_create_batch(ctypes.cast(self._cdescs, ctypes.c_void_p), self.n,
                                           ctypes.byref(self._mh.c), self.log_cap,
                                           ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                           _stream_ptr(stream), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.akmc_destroy_batch(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def compute_rates(self, stream=None):
        _check(self._lib.akmc_compute_rates(self._h, _stream_ptr(stream)))

    def step(self, n_events, stream=None):
        """Run n_events further events per voxel: a scalar or one per voxel (host),
        or a contiguous CUDA int64 tensor of one count per voxel (device)."""
        import torch
        if isinstance(n_events, torch.Tensor):
            if not (n_events.is_cuda and n_events.dtype == torch.int64 and n_events.is_contiguous()
                    and n_events.numel() == self.n):
                raise AkmcError(EINVAL, "device targets must be a contiguous CUDA int64 tensor of n_voxels entries")
            _check(self._lib.akmc_step_n(self._h, ctypes.c_void_p(n_events.data_ptr()), _stream_ptr(stream)))
            return
        arr = np.ascontiguousarray(np.broadcast_to(np.asarray(n_events, np.uint64), (self.n,)))
        _check(self._lib.akmc_step_n(self._h, _ptr(arr), _stream_ptr(stream)))

    def step_sublattice(self, voxel, superstep0, n_supersteps, sector_cells, window, asynchronous=False,
                        stream=None):
        """Sublattice supersteps superstep0 .. superstep0+n-1 of one voxel: one launch per
        superstep, or (asynchronous=True) one launch with per-sector readiness."""
        fn = self._lib.akmc_step_sublattice_async if asynchronous else self._lib.akmc_step_sublattice
        _check(fn(self._h, int(voxel), int(superstep0), int(n_supersteps), int(sector_cells), float(window),
                  _stream_ptr(stream)))

    def test_sublattice_stall(self, voxel, n_supersteps, sector_cells, window, stall_sector, stream=None):
        """Failure-detection hook: one sector never reports readiness (the voxel ends AKMC_ETIMEOUT)."""
        _check(self._lib.akmc_test_sublattice_stall(self._h, int(voxel), int(n_supersteps), int(sector_cells),
                                                    float(window), int(stall_sector), _stream_ptr(stream)))

    def set_targets(self, n_events, stream=None):
        arr = np.ascontiguousarray(np.broadcast_to(np.asarray(n_events, np.uint64), (self.n,)))
        _check(self._lib.akmc_set_targets(self._h, _ptr(arr), _stream_ptr(stream)))

    def launch_step(self, stream=None):
        """Run the targets stored by set_targets (capturable in a CUDA graph)."""
        _check(self._lib.akmc_launch_step(self._h, _stream_ptr(stream)))

    def capture_step(self, n_events, stream=None):
        """A torch CUDA graph whose replay runs n_events more events per voxel."""
        import torch
        s = stream if stream is not None else torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        self.set_targets(n_events, stream=s)   # outside the capture: copies targets, sets launch attributes
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            self.launch_step(stream=s)
        return g

    def reset_voxels(self, slots, descs, stream=None):
        """Re-seed slots in place with new descriptors (same L, n_vac, model, precision)."""
        sl = np.ascontiguousarray(slots, np.int32)
        cd = make_descs(descs)
        _check(self._lib.akmc_reset_voxels(self._h, _ptr(sl), ctypes.cast(cd, ctypes.c_void_p), int(sl.size),
                                           _stream_ptr(stream)))
        for s_, d in zip(sl.tolist(), descs):
            self.descs[s_] = d

    def set_launch(self, warps: int, ctas_per_sm: int = 0):
        _check(self._lib.akmc_set_launch(self._h, int(warps), int(ctas_per_sm)))

    def read_state(self, voxel: int, species=True, log=False, stream=None):
        d = self.descs[voxel]
        nv, N = int(d.n_vac), 2 * int(d.L) ** 3
        sp = np.empty(N, np.uint8) if species else None
        pos = np.empty(nv, np.int32)
        disp = np.empty(3 * nv, np.int32)
        rates = np.empty(8 * nv, np.float64)
        de = np.empty(8 * nv, np.float64)
        lg = np.empty(self.log_cap, np.int32) if (log and self.log_cap) else None
        st = StateC()
        st.species, st.vac_pos, st.vac_disp = (sp.ctypes.data if sp is not None else None), pos.ctypes.data, \
            disp.ctypes.data
        st.rates, st.dE = rates.ctypes.data, de.ctypes.data
        st.event_log = lg.ctypes.data if lg is not None else None
        _check(self._lib.akmc_read_state(self._h, int(voxel), ctypes.byref(st), _stream_ptr(stream)))
        return dict(species=sp, vac_pos=pos, vac_disp=disp.reshape(nv, 3), rates=rates.reshape(nv, 8),
                    dE=de.reshape(nv, 8), t_hi=st.t_hi, t_lo=st.t_lo, n_events=int(st.n_events),
                    status=int(st.status), event_log=lg)

    def load_state(self, voxel, species, vac_pos, t_hi=0.0, t_lo=0.0, n_events=0, stream=None):
        sp = np.ascontiguousarray(species, np.uint8)
        vp = np.ascontiguousarray(vac_pos, np.int32)
        _check(self._lib.akmc_load_state(self._h, int(voxel), _ptr(sp), _ptr(vp), float(t_hi), float(t_lo),
                                         int(n_events), _stream_ptr(stream)))

    @property
    def n_sites_total(self) -> int:
        return int(self._lib.akmc_batch_sites(self._h))

    @property
    def n_vac_total(self) -> int:
        return int(self._lib.akmc_batch_vacancies(self._h))

    def load_batch_state(self, species, vac_pos, t_hi=None, t_lo=None, n_events=None, stream=None):
        """Stream-ordered whole-batch load from host arrays (concatenated in
        voxel order); numpy arrays must stay alive until the stream passes."""
        def p(a, dt):
            if a is None:
                return None
            assert a.dtype == dt and a.flags.c_contiguous
            return ctypes.c_void_p(a.ctypes.data)
        _check(self._lib.akmc_load_batch_state(self._h, p(species, np.uint8), p(vac_pos, np.int32),
                                               p(t_hi, np.float64), p(t_lo, np.float64),
                                               p(n_events, np.uint64), _stream_ptr(stream)))

    def read_batch_state(self, out, stream=None):
        """Stream-ordered whole-batch read into the host arrays of `out`
        (keys species, vac_pos, vac_disp, t_hi, t_lo, n_events, status)."""
        def p(k):
            a = out.get(k)
            return ctypes.c_void_p(a.ctypes.data) if a is not None else None
        _check(self._lib.akmc_read_batch_state(self._h, p("species"), p("vac_pos"), p("vac_disp"), p("t_hi"),
                                               p("t_lo"), p("n_events"), p("status"), _stream_ptr(stream)))

    def host_buffers(self, pinned=True):
        """Host arrays sized for read/load_batch_state (pinned through torch)."""
        import torch

        def arr(n, dt):
            t = torch.empty(int(n), dtype=dt, pin_memory=pinned)
            return t.numpy(), t
        keep = []
        out = {}
        for k, n, dt in (("species", self.n_sites_total, torch.uint8), ("vac_pos", self.n_vac_total, torch.int32),
                         ("vac_disp", 3 * self.n_vac_total, torch.int32), ("t_hi", self.n, torch.float64),
                         ("t_lo", self.n, torch.float64), ("n_events", self.n, torch.int64),
                         ("status", self.n, torch.int32)):
            a, t = arr(n, dt)
            keep.append(t)
            out[k] = a.view(np.uint64) if k == "n_events" else a
        out["_keep"] = keep
        return out

    def sync_status(self, stream=None):
        per = np.zeros(self.n, np.int32)
        st = self._lib.akmc_sync_status(self._h, _stream_ptr(stream), _ptr(per))
        if st == ECUDA:
            _check(st)
        return int(st), per

    def read_density(self, voxel, stream=None):
        """EAM site densities of one voxel (int32, unit 2^-24), site order."""
        L = self.descs[voxel].L
        rho = np.zeros(2 * L ** 3, np.int32)
        _check(self._lib.akmc_read_density(self._h, int(voxel), _ptr(rho), _stream_ptr(stream)))
        return rho

    def workload_proxy(self, stream=None):
        """Eq. 10 workload proxy of every voxel from its current rates:
        (W, M_hat, E_hat) arrays, W = Gamma_tot / nu = M_hat exp(-E_hat / kT)."""
        W, M, E = (np.zeros(self.n, np.float64) for _ in range(3))
        _check(self._lib.akmc_workload_proxy(self._h, _ptr(W), _ptr(M), _ptr(E), _stream_ptr(stream)))
        return W, M, E

    def cluster_hist(self, voxel, mode=0, stream=None):
        h = np.zeros(8, np.int64)
        _check(self._lib.akmc_cluster_hist(self._h, int(voxel), int(mode), _ptr(h), _stream_ptr(stream)))
        return h


class SelectPlan:
    """Work plan and device scratch of the global masked softmax sampler for
    one segmentation (CSR offsets of the systems' concatenated logits)."""

    def __init__(self, offsets, device=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("akmc needs a CUDA device; there is no CPU fallback")
        lib = load_library()
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.n_seg = int(self.offsets.size - 1)
        nbytes = lib.akmc_select_scratch_bytes(_ptr(self.offsets), self.n_seg)
        if nbytes == 0:
            raise AkmcError(EINVAL, "invalid segment offsets")
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.scratch = torch.empty(int(nbytes), dtype=torch.uint8, device=dev)
        n_parts = ctypes.c_int32()
        _check(lib.akmc_select_plan(_ptr(self.offsets), self.n_seg, ctypes.c_void_p(self.scratch.data_ptr()),
                                    int(nbytes), ctypes.byref(n_parts), _stream_ptr(stream)))
        self.n_parts = int(n_parts.value)
        self.device = dev


def select_logits(plan, logits, tau=1.0, seed=0, counter=0, mask=None, out_index=None, out_logp=None,
                  stream=None):
    """Draw one logit per segment from softmax(z/tau) over the admissible logits
    (Eq. 1-2).  logits: float32 CUDA tensor covering the plan's offsets; mask:
    optional uint8 CUDA tensor of the same length.  Returns (index, logp) CUDA
    tensors (int64 offset within the segment or -1; float32 log-probability)."""
    import torch
    lib = load_library()
    if logits.dtype != torch.float32 or not logits.is_cuda or not logits.is_contiguous():
        raise AkmcError(EINVAL, "logits must be a contiguous float32 CUDA tensor")
    if logits.numel() < int(plan.offsets[-1]):
        raise AkmcError(EINVAL, "logits shorter than the plan's offsets")
    if mask is not None and (mask.dtype != torch.uint8 or not mask.is_cuda or mask.numel() < logits.numel()):
        raise AkmcError(EINVAL, "mask must be a uint8 CUDA tensor as long as the logits")
    if out_index is None:
        out_index = torch.empty(plan.n_seg, dtype=torch.int64, device=logits.device)
    if out_logp is None:
        out_logp = torch.empty(plan.n_seg, dtype=torch.float32, device=logits.device)
    _check(lib.akmc_select_logits(ctypes.c_void_p(logits.data_ptr()),
                                  ctypes.c_void_p(mask.data_ptr()) if mask is not None else None,
                                  plan.n_seg, plan.n_parts, float(tau), int(seed) & (2 ** 64 - 1),
                                  int(counter) & (2 ** 64 - 1), ctypes.c_void_p(plan.scratch.data_ptr()),
                                  ctypes.c_void_p(out_index.data_ptr()), ctypes.c_void_p(out_logp.data_ptr()),
                                  _stream_ptr(stream)))
    return out_index, out_logp
