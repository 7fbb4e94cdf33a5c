"""Python binding of the fm C ABI (``include/fm.h``): argument marshalling only.

Every step of a trajectory runs in ``libfm.so``.  PyTorch provides the device
workspace and the CUDA stream.  Importing this module loads the library and
raises if it is missing: there is no fallback implementation.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfm.so")

FM_OK, FM_EINVAL, FM_ENOMEM, FM_ECUDA, FM_ENUMERIC, FM_ETIMEOUT, FM_ESTATE = range(7)
FM_PROJECTIVE, FM_HOMODYNE, FM_HOMODYNE_RK4, FM_PROJECTIVE_POISSON = 0, 1, 2, 3
FM_FP64, FM_MIXED = 0, 1
FM_PROP_DENSE, FM_PROP_BANDED = 0, 1
FM_EE_FULL, FM_EE_SKETCH, FM_EE_AUTO = 0, 1, 2
FM_TILE_BN_AUTO, FM_TILE_BN_128, FM_TILE_BN_256 = 0, 1, 2
FM_TILE_CHOL_CHAINS = 1 << 7
FM_NOALLOC_MAX_SITES, FM_NOALLOC_MAX_N = 1024, 512


def FM_TILE_GROUP(g):
    """Raster groups of 2^(g+1) row tiles (fm_params.tile_config bits 2-4)."""
    return g << 2


def FM_TILE_DRAIN(d):
    """First-pass accumulators drained every 2^(d+1) K-blocks (fm_params.tile_config bits 5-6)."""
    return d << 5
PHASES = ("propagate", "measure", "gram", "cholesky", "trmm", "entropy")
FM_NPHASES = len(PHASES)
STATUS_NAMES = {0: "FM_OK", 1: "FM_EINVAL", 2: "FM_ENOMEM", 3: "FM_ECUDA", 4: "FM_ENUMERIC",
                5: "FM_ETIMEOUT", 6: "FM_ESTATE"}


class fm_params(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int32), ("Ly", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("protocol", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("reorth_interval", ctypes.c_int32), ("event_capacity", ctypes.c_int32),
                ("tile_config", ctypes.c_int32), ("J", ctypes.c_double), ("dt", ctypes.c_double),
                ("gamma", ctypes.c_double), ("seed", ctypes.c_uint64), ("traj_id", ctypes.c_uint64)]


class fm_event(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("traj", ctypes.c_int32), ("site", ctypes.c_int32),
                ("u", ctypes.c_double), ("p", ctypes.c_double), ("outcome", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class fm_tuning(ctypes.Structure):
    _fields_ = [("tile_config", ctypes.c_int32), ("reorth_interval", ctypes.c_int32),
                ("ms_per_step", ctypes.c_double), ("ortho_err", ctypes.c_double),
                ("tried", ctypes.c_int32), ("rejected", ctypes.c_int32), ("ortho_mid", ctypes.c_double)]


class FmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, code), msg))
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libfm.so is not built (run __graft_entry__.build()); "
                          "this package has no non-CUDA fallback")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp, i32, i64, u64, dbl, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, \
        ctypes.c_double, ctypes.c_size_t
    sigs = {
        "fm_workspace_bytes": (sz, [P(fm_params)]),
        "fm_init_state": (i32, [P(fm_params), vp, sz, vp, P(vp)]),
        "fm_step": (i32, [vp, i32]),
        "fm_set_gammas": (i32, [vp, P(dbl)]),
        "fm_reset_trajectory": (i32, [vp, i32, u64, dbl]),
        "fm_steps_done": (i32, [vp, i32, P(i64)]),
        "fm_entropy": (i32, [vp, i32, P(i32), i32, P(dbl)]),
        "fm_mutual_info": (i32, [vp, i32, P(i32), i32, P(i32), i32, P(dbl)]),
        "fm_entropy_async": (i32, [vp, i32, P(i32), i32, P(i64)]),
        "fm_entropy_wait": (i32, [vp, i64, P(dbl)]),
        "fm_entropy_ready": (i32, [vp, i64, P(i32)]),
        "fm_copy_U": (i32, [vp, i32, vp, i64]),
        "fm_set_U": (i32, [vp, i32, vp, i64]),
        "fm_occupations": (i32, [vp, i32, P(dbl)]),
        "fm_orthonormality_error": (i32, [vp, i32, P(i32), i32, P(dbl)]),
        "fm_take_events": (i32, [vp, P(fm_event), i32, P(i32), P(i64)]),
        "fm_save": (i32, [vp, ctypes.c_char_p]),
        "fm_load": (i32, [vp, ctypes.c_char_p]),
        "fm_kernel_launches": (i64, [vp]),
        "fm_set_timing": (i32, [vp, i32]),
        "fm_set_graphs": (i32, [vp, i32]),
        "fm_phase_times": (i32, [vp, P(dbl), P(i64)]),
        "fm_last_error": (ctypes.c_char_p, [vp]),
        "fm_destroy": (None, [vp]),
        "fm_version": (ctypes.c_char_p, []),
        "fm_entropy_noalloc": (i32, [vp, i32, i32, P(i32), i32, vp, vp]),
        "fm_autotune": (i32, [P(fm_params), vp, sz, vp, i32, i32, dbl, i32, P(fm_tuning)]),
        "fm_density_correlation": (i32, [vp, i32, P(dbl)]),
        "fm_set_propagation": (i32, [vp, i32]),
        "fm_particle_covariance": (i32, [vp, i32, P(i32), i32, P(i32), i32, P(dbl)]),
        "fm_set_entropy_method": (i32, [vp, i32]),
        "fm_entropy_sketch_info": (i32, [vp, P(i32), P(dbl), P(i32)]),
        "fm_reorth_stats": (i32, [vp, P(i64), P(i64), P(dbl)]),
        "fm_force_outcomes": (i32, [vp, P(fm_event), i32]),
        "fm_group_create": (i32, [P(vp), i32, vp, P(vp)]),
        "fm_group_step": (i32, [vp, i32]),
        "fm_group_period": (i32, [vp]),
        "fm_group_last_error": (ctypes.c_char_p, [vp]),
        "fm_group_destroy": (None, [vp]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _i32_array(x):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.int32).ravel())
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def make_params(Lx, Ly=1, batch=1, protocol=FM_PROJECTIVE, precision=FM_FP64, reorth_interval=1,
                event_capacity=0, J=1.0, dt=0.05, gamma=0.5, seed=0, traj_id=0, tile_config=0):
    return fm_params(Lx=Lx, Ly=Ly, batch=batch, protocol=protocol, precision=precision,
                     reorth_interval=reorth_interval, event_capacity=event_capacity, tile_config=tile_config,
                     J=J, dt=dt, gamma=gamma, seed=seed, traj_id=traj_id)


def fm_workspace_bytes(params):
    return int(lib.fm_workspace_bytes(ctypes.byref(params)))


def fm_version():
    return lib.fm_version().decode()


def fm_entropy_noalloc(d_U, L, N, sites, d_S, stream=None):
    """S_A of a device complex128 U (L x N, column-major) into the device double d_S; no allocation.

    d_U and d_S are device pointers (ints); stream a cudaStream_t handle or None.
    Returns the status code.
    """
    a, p = _i32_array(sites)
    return int(lib.fm_entropy_noalloc(ctypes.c_void_p(d_U), int(L), int(N), p, int(a.size), ctypes.c_void_p(d_S),
                                      ctypes.c_void_p(stream)))


def autotune(params, steps=4, max_reorth=4, ortho_tol=1e-6, use_graphs=True, device="cuda", stream=None):
    """fm_autotune on a scratch workspace; returns a dict of the chosen settings and their measurements."""
    import torch
    nbytes = fm_workspace_bytes(params)
    if nbytes == 0:
        raise FmError(FM_EINVAL, "invalid parameters")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
    if stream is None:
        stream = torch.cuda.current_stream(ws.device)
    out = fm_tuning()
    code = lib.fm_autotune(ctypes.byref(params), ctypes.c_void_p(ws.data_ptr()), nbytes,
                           ctypes.c_void_p(stream.cuda_stream), int(steps), int(max_reorth), float(ortho_tol),
                           1 if use_graphs else 0, ctypes.byref(out))
    del ws
    if code != FM_OK:
        raise FmError(code, "fm_autotune failed")
    return {"tile_config": out.tile_config, "reorth_interval": out.reorth_interval,
            "ms_per_step": out.ms_per_step, "ortho_err": out.ortho_err, "ortho_mid": out.ortho_mid,
            "tried": out.tried, "rejected": out.rejected}


class Trajectories:
    """A batch of trajectories held on the GPU (one ``fm_state``).

    The device workspace is a torch uint8 tensor owned by this object; work is
    issued on the torch stream current at construction.
    """

    def __init__(self, params, device="cuda", stream=None):
        import torch
        self.params = params
        self.L = params.Lx * params.Ly
        self.N = self.L // 2
        self.batch = params.batch
        nbytes = fm_workspace_bytes(params)
        if nbytes == 0:
            raise FmError(FM_EINVAL, "invalid parameters")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        if stream is None:
            stream = torch.cuda.current_stream(self.workspace.device)
        self.stream = stream
        handle = ctypes.c_void_p()
        code = lib.fm_init_state(ctypes.byref(params), ctypes.c_void_p(self.workspace.data_ptr()),
                                 ctypes.c_size_t(nbytes), ctypes.c_void_p(stream.cuda_stream),
                                 ctypes.byref(handle))
        if code != FM_OK:
            raise FmError(code, "fm_init_state failed")
        self._h = handle

    # -- marshalling helpers
    def _check(self, code):
        if code != FM_OK:
            raise FmError(code, lib.fm_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib.fm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C ABI, same names without the prefix
    def step(self, nsteps=1):
        self._check(lib.fm_step(self._h, int(nsteps)))

    def set_gammas(self, gammas):
        g = np.ascontiguousarray(np.asarray(gammas, dtype=np.float64))
        assert g.size == self.batch
        self._check(lib.fm_set_gammas(self._h, g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def reset_trajectory(self, b, traj_id, gamma):
        self._check(lib.fm_reset_trajectory(self._h, int(b), int(traj_id), float(gamma)))

    def steps_done(self, b=0):
        out = ctypes.c_int64()
        self._check(lib.fm_steps_done(self._h, int(b), ctypes.byref(out)))
        return out.value

    def entropy(self, sites, b=0):
        a, p = _i32_array(sites)
        out = ctypes.c_double()
        self._check(lib.fm_entropy(self._h, int(b), p, int(a.size), ctypes.byref(out)))
        return out.value

    def entropy_async(self, sites, b=0):
        """Start S_A of trajectory b at this point of the step sequence; returns a ticket."""
        a, p = _i32_array(sites)
        t = ctypes.c_int64()
        self._check(lib.fm_entropy_async(self._h, int(b), p, int(a.size), ctypes.byref(t)))
        return t.value

    def entropy_wait(self, ticket):
        out = ctypes.c_double()
        self._check(lib.fm_entropy_wait(self._h, int(ticket), ctypes.byref(out)))
        return out.value

    def entropy_ready(self, ticket):
        """True if entropy_wait(ticket) would return at once."""
        out = ctypes.c_int32()
        self._check(lib.fm_entropy_ready(self._h, int(ticket), ctypes.byref(out)))
        return bool(out.value)

    def mutual_info(self, A, B, b=0):
        a, pa = _i32_array(A)
        c, pb = _i32_array(B)
        out = ctypes.c_double()
        self._check(lib.fm_mutual_info(self._h, int(b), pa, int(a.size), pb, int(c.size), ctypes.byref(out)))
        return out.value

    def set_entropy_method(self, method):
        """FM_EE_FULL (eigenvalues of C_A), FM_EE_SKETCH (cross-block sketch) or FM_EE_AUTO
        (the sketch from 1024 sites on), the last two for mixed precision."""
        self._check(lib.fm_set_entropy_method(self._h, int(method)))

    def entropy_sketch_info(self):
        """(rank, check, fell_back) of the last synchronous sketch entropy."""
        r, f = ctypes.c_int32(), ctypes.c_int32()
        c = ctypes.c_double()
        self._check(lib.fm_entropy_sketch_info(self._h, ctypes.byref(r), ctypes.byref(c), ctypes.byref(f)))
        return r.value, c.value, bool(f.value)

    def set_propagation(self, mode):
        """FM_PROP_DENSE (dense GEMM) or FM_PROP_BANDED (stencils of the circulant propagator)."""
        self._check(lib.fm_set_propagation(self._h, int(mode)))

    def density_correlation(self, b=0):
        """c[d] of Eq. (2) per displacement d = dx + Lx dy (numpy array of L floats, c[0] = 0)."""
        out = np.empty(self.L, dtype=np.float64)
        self._check(lib.fm_density_correlation(self._h, int(b), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def particle_covariance(self, A, B, b=0):
        """G_AB of Eq. (GAB) on the lattice for disjoint site lists A and B."""
        a, pa = _i32_array(A)
        c, pb = _i32_array(B)
        out = ctypes.c_double()
        self._check(lib.fm_particle_covariance(self._h, int(b), pa, int(a.size), pb, int(c.size), ctypes.byref(out)))
        return out.value

    def copy_U(self, b=0):
        U = np.empty((self.L, self.N), dtype=np.complex128, order="F")
        self._check(lib.fm_copy_U(self._h, int(b), ctypes.c_void_p(U.ctypes.data), self.L))
        return U

    def set_U(self, U, b=0):
        U = np.asfortranarray(np.asarray(U, dtype=np.complex128))
        assert U.shape == (self.L, self.N)
        self._check(lib.fm_set_U(self._h, int(b), ctypes.c_void_p(U.ctypes.data), self.L))

    def occupations(self, b=0, out=None):
        n = np.empty(self.L, dtype=np.float64) if out is None else out
        assert n.dtype == np.float64 and n.size == self.L and n.flags.c_contiguous
        self._check(lib.fm_occupations(self._h, int(b), n.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return n

    def orthonormality_error(self, cols, b=0):
        a, p = _i32_array(cols)
        out = ctypes.c_double()
        self._check(lib.fm_orthonormality_error(self._h, int(b), p, int(a.size), ctypes.byref(out)))
        return out.value

    def take_events(self, cap=1 << 20):
        buf = (fm_event * cap)()
        count = ctypes.c_int32()
        dropped = ctypes.c_int64()
        self._check(lib.fm_take_events(self._h, buf, cap, ctypes.byref(count), ctypes.byref(dropped)))
        ev = [(buf[i].traj, buf[i].step, buf[i].site, buf[i].u, buf[i].p, buf[i].outcome)
              for i in range(count.value)]
        return ev, dropped.value

    def force_outcomes(self, events):
        """Replay: events as (traj, step, site, outcome) tuples (the first, second, third and last
        fields of take_events() entries also fit); an empty list clears the replay."""
        events = list(events)
        buf = (fm_event * max(1, len(events)))()
        for i, e in enumerate(events):
            buf[i].traj, buf[i].step, buf[i].site, buf[i].outcome = int(e[0]), int(e[1]), int(e[2]), int(e[-1])
        self._check(lib.fm_force_outcomes(self._h, buf, len(events)))

    def save(self, path):
        self._check(lib.fm_save(self._h, str(path).encode()))

    def load(self, path):
        self._check(lib.fm_load(self._h, str(path).encode()))

    def set_graphs(self, enable=True):
        self._check(lib.fm_set_graphs(self._h, 1 if enable else 0))

    def set_timing(self, enable=True):
        self._check(lib.fm_set_timing(self._h, 1 if enable else 0))

    def phase_times(self):
        """{phase: (milliseconds, launches)} accumulated since the last call."""
        ms = (ctypes.c_double * len(PHASES))()
        cnt = (ctypes.c_int64 * len(PHASES))()
        self._check(lib.fm_phase_times(self._h, ms, cnt))
        return {name: (ms[i], cnt[i]) for i, name in enumerate(PHASES)}

    def reorth_stats(self):
        """Second-pass guard of the mixed path: (checks, extra_passes, [d2, o2, d3, o3]) -- the
        largest diagonal / off-diagonal |U^dag U - 1| measured by the second passes and the extra
        passes since the previous call."""
        c, e = ctypes.c_int64(), ctypes.c_int64()
        mx = (ctypes.c_double * 4)()
        self._check(lib.fm_reorth_stats(self._h, ctypes.byref(c), ctypes.byref(e), mx))
        return c.value, e.value, list(mx)

    @property
    def kernel_launches(self):
        return int(lib.fm_kernel_launches(self._h))

    def last_error(self):
        return lib.fm_last_error(self._h).decode()


class Group:
    """Several Trajectories objects advanced together by one CUDA graph (fm_group_*)."""

    def __init__(self, members, stream=None):
        import torch
        self.members = list(members)              # keep the states alive
        arr = (ctypes.c_void_p * len(self.members))(*[m._h.value for m in self.members])
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        code = lib.fm_group_create(arr, len(self.members), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if code != FM_OK:
            raise FmError(code, "fm_group_create failed")
        self._h = h

    @property
    def period(self):
        return int(lib.fm_group_period(self._h))

    def step(self, nsteps):
        code = lib.fm_group_step(self._h, int(nsteps))
        if code != FM_OK:
            raise FmError(code, lib.fm_group_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib.fm_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
