"""TEST INFRASTRUCTURE ONLY: ctypes binding of the serial float64 AKMC oracle.

The oracle (akmc_oracle.cpp) is a plain, slow, obviously correct C++
implementation of rejection-free vacancy AKMC.  Only tests/, the smoke check
and the CPU-baseline leg of bench.py may import this package; the CUDA
library never does, and this package never imports the CUDA library.
Inputs (models, voxel descriptors, lattices) come from synth/.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "akmc_oracle.cpp")
_HDR = os.path.join(_HERE, "akmc_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ETRAPPED, ENUMERIC = 0, 1, 5, 6


def build(force: bool = False) -> str:
    """Compile the oracle with plain IEEE semantics (no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH) or
             os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-Wall", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Model(ctypes.Structure):
    _fields_ = [("eps1", ctypes.c_double * 25), ("eps2", ctypes.c_double * 25),
                ("E0", ctypes.c_double * 4), ("nu", ctypes.c_double), ("a", ctypes.c_double),
                ("r_cut", ctypes.c_double), ("n_r", ctypes.c_int32), ("n_rho", ctypes.c_int32),
                ("rho_h", ctypes.c_double), ("phi_tab", ctypes.c_void_p),
                ("f_tab", ctypes.c_void_p), ("F_tab", ctypes.c_void_p)]


class _Desc(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("n_vac", ctypes.c_int32), ("frac", ctypes.c_double * 3),
                ("T", ctypes.c_double), ("model", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("uid", ctypes.c_uint64)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P, D, I, U64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_uint64
            sig = {
                "orc_create": (P, [ctypes.POINTER(_Desc), ctypes.POINTER(_Model), ctypes.POINTER(I)]),
                "orc_destroy": (None, [P]),
                "orc_load": (I, [P, P, P, ctypes.c_int32, D, D, U64]),
                "orc_step": (I, [P, U64, P, P]),
                "orc_get": (I, [P, P, P, P, P, P, P, P, P]),
                "orc_n_sites": (ctypes.c_int32, [P]),
                "orc_n_vac": (ctypes.c_int32, [P]),
                "orc_total_rate": (D, [P]),
                "orc_energy": (D, [P]),
                "orc_hop_de_local": (D, [P, I, I]),
                "orc_hop_de_brute": (D, [P, I, I]),
                "orc_hop_rate": (D, [P, I, I]),
                "orc_rho_fixed": (ctypes.c_int64, [P, I]),
                "orc_rho_all": (None, [P, P]),
                "orc_step_sublattice": (I, [P, U64, ctypes.c_uint32, ctypes.c_int32, D, ctypes.c_int32, P]),
                "orc_set_debug": (None, [P, I]),
                "orc_debug_counts": (None, [P, P]),
                "orc_tracer_r2": (D, [P]),
                "orc_cluster_hist": (ctypes.c_int32, [P, I, P, P]),
                "orc_shell_constants": (I, [ctypes.POINTER(_Model), P, P]),
                "orc_embed": (D, [ctypes.POINTER(_Model), I, ctypes.c_int64, ctypes.POINTER(I)]),
                "orc_philox4x32_10": (None, [P, P, P]),
                "orc_event_uniforms": (None, [U64, U64, U64, ctypes.POINTER(D), ctypes.POINTER(D)]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class _ModelHolder:
    """Keeps the numpy tables alive while the C struct points at them."""

    def __init__(self, model):
        m = _Model()
        m.eps1[:] = [float(x) for x in np.asarray(model.eps1, dtype=np.float64).ravel()]
        m.eps2[:] = [float(x) for x in np.asarray(model.eps2, dtype=np.float64).ravel()]
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


class Voxel:
    """One oracle voxel (owns the C object)."""

    def __init__(self, desc, model):
        self._mh = _ModelHolder(model)
        d = _Desc()
        d.L, d.n_vac = int(desc.L), int(desc.n_vac)
        fr = list(desc.frac) + [0.0] * (3 - len(desc.frac))
        d.frac[:] = [float(x) for x in fr[:3]]
        d.T, d.model = float(desc.T), int(desc.model)
        d.seed, d.uid = int(desc.seed), int(desc.uid)
        st = ctypes.c_int(0)
        self._lib = lib()
        self._h = self._lib.orc_create(ctypes.byref(d), ctypes.byref(self._mh.c), ctypes.byref(st))
        if not self._h:
            raise ValueError("oracle rejected the voxel descriptor (status %d)" % st.value)
        self.status = st.value
        self.L = int(desc.L)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    @property
    def n_sites(self):
        return int(self._lib.orc_n_sites(self._h))

    @property
    def n_vac(self):
        return int(self._lib.orc_n_vac(self._h))

    def load(self, species, vac_pos, t_hi=0.0, t_lo=0.0, n_events=0):
        sp = np.ascontiguousarray(species, dtype=np.uint8)
        vp = np.ascontiguousarray(vac_pos, dtype=np.int32)
        assert sp.size == self.n_sites
        st = self._lib.orc_load(self._h, _ptr(sp), _ptr(vp), int(vp.size), float(t_hi), float(t_lo),
                                int(n_events))
        if st == EINVAL:
            raise ValueError("oracle rejected the state")
        self.status = st
        return st

    def step(self, n, log=False, dt=False):
        buf = np.full(int(n), -1, dtype=np.int32) if log else None
        dts = np.full(int(n), np.nan, dtype=np.float64) if dt else None
        self.status = self._lib.orc_step(self._h, int(n), _ptr(buf), _ptr(dts))
        if dt:
            return buf, dts
        return buf

    def state(self):
        nv, N = self.n_vac, self.n_sites
        sp = np.empty(N, np.uint8)
        pos = np.empty(nv, np.int32)
        disp = np.empty(3 * nv, np.int32)
        rates = np.empty(8 * nv, np.float64)
        de = np.empty(8 * nv, np.float64)
        th, tl = ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_uint64()
        st = self._lib.orc_get(self._h, _ptr(sp), _ptr(pos), _ptr(disp), _ptr(rates), _ptr(de),
                               ctypes.byref(th), ctypes.byref(tl), ctypes.byref(n))
        return dict(species=sp, vac_pos=pos, vac_disp=disp.reshape(nv, 3), rates=rates.reshape(nv, 8),
                    dE=de.reshape(nv, 8), t_hi=th.value, t_lo=tl.value, n_events=n.value, status=st)

    def total_rate(self):
        return float(self._lib.orc_total_rate(self._h))

    def energy(self):
        return float(self._lib.orc_energy(self._h))

    def hop_de_local(self, slot, d):
        return float(self._lib.orc_hop_de_local(self._h, slot, d))

    def hop_de_brute(self, slot, d):
        return float(self._lib.orc_hop_de_brute(self._h, slot, d))

    def hop_rate(self, slot, d):
        return float(self._lib.orc_hop_rate(self._h, slot, d))

    def rho_fixed(self, site):
        return int(self._lib.orc_rho_fixed(self._h, int(site)))

    def step_sublattice(self, k0, n_supersteps, sector_cells, window, reverse=False):
        """Synchronous sublattice supersteps k0 .. k0+n-1; returns the events made per superstep."""
        ev = np.zeros(int(n_supersteps), np.uint64)
        st = self._lib.orc_step_sublattice(self._h, int(k0), int(n_supersteps), int(sector_cells), float(window),
                                           int(bool(reverse)), _ptr(ev))
        if st == EINVAL:
            raise ValueError("bad sublattice parameters")
        self.status = st
        return ev

    def rho_all(self):
        out = np.zeros(self.n_sites, np.int64)
        self._lib.orc_rho_all(self._h, _ptr(out))
        return out

    def set_debug(self, flags):
        self._lib.orc_set_debug(self._h, int(flags))

    def debug_counts(self):
        out = np.zeros(5, np.uint64)
        self._lib.orc_debug_counts(self._h, _ptr(out))
        return dict(rate_mismatch=int(out[0]), declared_ties=int(out[1]), scan_disagree=int(out[2]),
                    rho_mismatch=int(out[3]), checked=int(out[4]))

    def tracer_r2(self):
        return float(self._lib.orc_tracer_r2(self._h))

    def cluster_hist(self, mode=0):
        hist = np.zeros(8, np.int64)
        sizes = np.zeros(self.n_sites, np.int32)
        nc = self._lib.orc_cluster_hist(self._h, int(mode), _ptr(hist), _ptr(sizes))
        return hist, sizes[:nc].copy()


def shell_constants(model):
    mh = _ModelHolder(model)
    phi = np.zeros(50, np.float64)
    fq = np.zeros(20, np.int64)
    st = lib().orc_shell_constants(ctypes.byref(mh.c), _ptr(phi), _ptr(fq))
    if st:
        raise ValueError("bad EAM tables")
    return phi.reshape(10, 5), fq.reshape(4, 5)


def embed(model, species, rho_fixed):
    mh = _ModelHolder(model)
    err = ctypes.c_int(0)
    v = lib().orc_embed(ctypes.byref(mh.c), int(species), int(rho_fixed), ctypes.byref(err))
    return float(v), int(err.value)


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return [int(x) for x in out]


def event_uniforms(seed, uid, n):
    u1, u2 = ctypes.c_double(), ctypes.c_double()
    lib().orc_event_uniforms(int(seed), int(uid), int(n), ctypes.byref(u1), ctypes.byref(u2))
    return u1.value, u2.value


def _ensemble_worker(args):
    desc, model, n_events, mode, start = args
    v = Voxel(desc, model)
    if start is not None:
        v.load(*start)
    h0 = v.cluster_hist(mode)[0]
    v.step(n_events)
    return h0, v.cluster_hist(mode)[0], int(v.status)


def ensemble_cluster_hist(descs, model, n_events, mode=0, procs=None, start=None):
    """Cu cluster histograms of independent oracle runs: each voxel starts from
    its seeded placement (or from `start` = (species, vac_pos), the same
    lattice for every voxel) and takes `n_events` events.  Returns (initial
    histograms, final histograms, statuses), one row per voxel.  Voxels run on
    `procs` spawned processes (never forked, so callers that already hold a
    CUDA context are safe)."""
    import multiprocessing as mp
    build()
    procs = max(1, min(len(descs), procs or os.cpu_count() or 1))
    jobs = [(d, model, int(n_events), int(mode), start) for d in descs]
    if procs == 1:
        res = [_ensemble_worker(j) for j in jobs]
    else:
        with mp.get_context("spawn").Pool(procs) as pool:
            res = pool.map(_ensemble_worker, jobs)
    return (np.array([r[0] for r in res]), np.array([r[1] for r in res]),
            np.array([r[2] for r in res]))
