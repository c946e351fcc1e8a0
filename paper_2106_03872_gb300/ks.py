"""Thin ctypes binding of the C ABI in include/ks.h (argument marshalling only).

Every compute step runs in the CUDA library ``libks_gb300.so``; loading fails loudly if
it has not been built (``python -c "import __graft_entry__ as g; g.build()"``).  There is
no CPU fallback.  The functions keep the C names; ``Grid`` is a small convenience wrapper
that owns a handle and marshals numpy arrays and torch device tensors.
"""
import ctypes as ct
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libks_gb300.so")

KS_OK, KS_ERR_ARG, KS_ERR_NOMEM, KS_ERR_NOT_POSDEF, KS_ERR_DIVERGED, KS_ERR_TIMEOUT, KS_ERR_CUDA, KS_PENDING, \
    KS_ERR_STATE = range(9)
STATUS_NAMES = ["KS_OK", "KS_ERR_ARG", "KS_ERR_NOMEM", "KS_ERR_NOT_POSDEF", "KS_ERR_DIVERGED", "KS_ERR_TIMEOUT",
                "KS_ERR_CUDA", "KS_PENDING", "KS_ERR_STATE"]
KS_FP64, KS_MIXED_BF16X3 = 0, 1
PRECISIONS = {"fp64": KS_FP64, "bf16x3": KS_MIXED_BF16X3}

# Every symbol declared in include/ks.h.
EXPORTS = ["ks_count_gvectors", "ks_grid_create", "ks_grid_destroy", "ks_grid_gvectors", "ks_grid_device_bytes",
           "ks_get_vloc", "ks_set_states", "ks_get_states", "ks_states_device", "ks_apply_h", "ks_apply_h_host",
           "ks_density", "ks_orthonormalize", "ks_rayleigh_ritz", "ks_block_iteration", "ks_block_iteration_pc", "ks_set_option", "ks_scf", "ks_td_step", "ks_td_step_dipole", "ks_kick", "ks_dipole", "ks_forces",
           "ks_set_positions", "ks_get_positions", "ks_ehrenfest",
           "ks_serve_create", "ks_serve_create_ex", "ks_serve_destroy", "ks_serve_submit", "ks_serve_poll", "ks_serve_result_info", "ks_serve_stats",
           "ks_profile", "ks_profile_read", "ks_profile_span", "ks_kernel_launches", "ks_tc_status_check", "ks_autotune_report", "ks_overlap_noalloc", "ks_last_error"]


KS_OPT_FP64_SUBSPACE = 1


class KsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status, msg))
        self.status = status


class CellDesc(ct.Structure):
    _fields_ = [("L", ct.c_double), ("N", ct.c_int), ("ecut", ct.c_double), ("natoms", ct.c_int),
                ("pos", ct.POINTER(ct.c_double)), ("vloc_depth", ct.c_double), ("vloc_width", ct.c_double),
                ("nproj", ct.c_int), ("proj_sigma", ct.c_double), ("proj_rc", ct.c_double),
                ("proj_D", ct.c_double), ("nstates", ct.c_int), ("occ", ct.POINTER(ct.c_double)),
                ("prec", ct.c_int)]


_lib = None


def load():
    """Load the built library (raises if missing: the product path has no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("CUDA library %s is not built; run paper_2106_03872_gb300.build.build()" % LIB_PATH)
    lib = ct.CDLL(LIB_PATH)
    P = ct.c_void_p
    dp = ct.POINTER(ct.c_double)
    ip = ct.POINTER(ct.c_int)
    sig = {
        "ks_count_gvectors": [ct.c_double, ct.c_int, ct.c_double, ip],
        "ks_grid_create": [ct.POINTER(CellDesc), ct.POINTER(P)],
        "ks_grid_destroy": [P],
        "ks_grid_gvectors": [P, ip, ip],
        "ks_grid_device_bytes": [P, ct.POINTER(ct.c_size_t)],
        "ks_get_vloc": [P, dp],
        "ks_set_states": [P, dp],
        "ks_get_states": [P, dp],
        "ks_states_device": [P, ct.POINTER(P)],
        "ks_apply_h": [P, P, P, ct.c_int, P],
        "ks_apply_h_host": [P, dp, dp, ct.c_int],
        "ks_density": [P, P, P],
        "ks_orthonormalize": [P, dp, P],
        "ks_rayleigh_ritz": [P, dp, P],
        "ks_block_iteration": [P, ct.c_int, dp, P],
        "ks_block_iteration_pc": [P, ct.c_int, ct.c_int, dp, P],
        "ks_scf": [P, ct.c_int, ct.c_int, ct.c_int, ct.c_double, ct.c_int, ct.c_double, dp, dp, ip, P],
        "ks_td_step": [P, ct.c_double, ct.c_int, ct.c_int, ct.c_int, dp, dp, P],
        "ks_td_step_dipole": [P, ct.c_double, ct.c_int, ct.c_int, ct.c_int, dp, dp, dp, P],
        "ks_kick": [P, dp, P],
        "ks_dipole": [P, dp, P],
        "ks_forces": [P, dp, P],
        "ks_set_positions": [P, dp, P],
        "ks_get_positions": [P, dp],
        "ks_ehrenfest": [P, ct.c_double, ct.c_int, ct.c_int, dp, dp, dp, dp, P],
        "ks_serve_create": [ct.c_size_t, ct.POINTER(P)],
        "ks_serve_destroy": [P],
        "ks_serve_submit": [P, ct.POINTER(CellDesc), dp, ct.c_int, ct.c_int, ct.c_double,
                            ct.POINTER(ct.c_uint64)],
        "ks_serve_poll": [P, ct.c_uint64, ct.c_int, dp, dp, dp],
        "ks_serve_result_info": [P, ct.c_uint64, ip, ip, ip],
        "ks_overlap_noalloc": [P, P, ct.c_int, ct.c_int, ct.c_int, ct.c_int, P, P],
        "ks_set_option": [P, ct.c_int, ct.c_int],
        "ks_tc_status_check": [ct.c_int],
        "ks_autotune_report": [ct.c_char_p, ct.c_size_t, ct.POINTER(ct.c_size_t)],
        "ks_serve_create_ex": [ct.c_size_t, ct.c_int, ct.POINTER(P)],
        "ks_serve_stats": [P, dp, ct.c_int],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ct.c_int
    lib.ks_profile.argtypes = [P, ct.c_int]
    lib.ks_profile.restype = ct.c_int
    lib.ks_profile_read.argtypes = [P, ct.c_int, ct.c_char_p, ct.c_int, dp, ct.POINTER(ct.c_long)]
    lib.ks_profile_read.restype = ct.c_int
    lib.ks_profile_span.argtypes = [P, ct.c_int, ct.c_char_p, ct.c_int, dp, dp]
    lib.ks_profile_span.restype = ct.c_int
    lib.ks_kernel_launches.argtypes = []
    lib.ks_kernel_launches.restype = ct.c_uint64
    lib.ks_last_error.argtypes = []
    lib.ks_last_error.restype = ct.c_char_p
    _lib = lib
    return lib


def check(status):
    if status != KS_OK:
        raise KsError(status, load().ks_last_error().decode())
    return status


def _dptr(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_double)) if a is not None else None


def make_desc(cell, prec="bf16x3", nstates=None, occ=None):
    """CellDesc from an input dict (see inputs.py); keeps the arrays alive on the struct."""
    pos = np.ascontiguousarray(np.asarray(cell["pos"], float).reshape(-1, 3))
    d = CellDesc()
    d.L, d.N, d.ecut = float(cell["L"]), int(cell["N"]), float(cell["ecut"])
    d.natoms = len(pos)
    d.pos = _dptr(pos)
    d.vloc_depth, d.vloc_width = float(cell["vloc_depth"]), float(cell["vloc_width"])
    d.nproj = int(cell["nproj"])
    d.proj_sigma, d.proj_rc, d.proj_D = float(cell["proj_sigma"]), float(cell["proj_rc"]), float(cell["proj_D"])
    d.nstates = int(nstates if nstates is not None else cell["nstates"])
    occ = cell.get("occ") if occ is None else occ
    occ_arr = None if occ is None else np.ascontiguousarray(np.asarray(occ, float))
    d.occ = _dptr(occ_arr)
    d.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    d._keep = (pos, occ_arr)
    return d


def overlap_noalloc(a_ptr, b_ptr, m, n, nG, fp64, out_ptr, stream=None):
    """out = A^H B ([m][n] complex128, device) without any device allocation (see ks.h)."""
    check(load().ks_overlap_noalloc(ct.c_void_p(a_ptr), ct.c_void_p(b_ptr), int(m), int(n), int(nG),
                                    1 if fp64 else 0, ct.c_void_p(out_ptr), _stream_ptr(stream)))


def autotune_report():
    """The autotuner's decisions so far (list of dicts: key, per-candidate ms, choice)."""
    import json
    n = ct.c_size_t(0)
    check(load().ks_autotune_report(None, 0, ct.byref(n)))
    buf = ct.create_string_buffer(max(1, n.value))
    check(load().ks_autotune_report(buf, n.value, ct.byref(n)))
    return json.loads(buf.value.decode() or "[]")


def kernel_launches():
    return int(load().ks_kernel_launches())


def count_gvectors(L, N, ecut):
    n = ct.c_int()
    check(load().ks_count_gvectors(L, N, ecut, ct.byref(n)))
    return n.value


def _stream_ptr(stream):
    if stream is None:
        return None
    return ct.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Grid:
    """Owns a ks_grid handle."""

    def __init__(self, cell, prec="bf16x3", nstates=None, occ=None):
        lib = load()
        self.desc = make_desc(cell, prec, nstates, occ)
        self.h = ct.c_void_p()
        check(lib.ks_grid_create(ct.byref(self.desc), ct.byref(self.h)))
        self.nstates = self.desc.nstates
        self.N = self.desc.N
        self.prec = self.desc.prec
        n = ct.c_int()
        check(lib.ks_grid_gvectors(self.h, ct.byref(n), None))
        self.nG = n.value

    def close(self):
        if self.h:
            check(load().ks_grid_destroy(self.h))
            self.h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- host-side queries
    def gvectors(self):
        m = np.zeros((self.nG, 3), dtype=np.int32)
        n = ct.c_int()
        check(load().ks_grid_gvectors(self.h, ct.byref(n), m.ctypes.data_as(ct.POINTER(ct.c_int))))
        return m

    def device_bytes(self):
        b = ct.c_size_t()
        check(load().ks_grid_device_bytes(self.h, ct.byref(b)))
        return b.value

    def vloc(self):
        v = np.zeros(self.N ** 3)
        check(load().ks_get_vloc(self.h, _dptr(v)))
        return v.reshape(self.N, self.N, self.N)

    def set_option(self, option, value):
        """KS_OPT_FP64_SUBSPACE (1): FP64 Cholesky and Rayleigh-Ritz on a mixed handle."""
        check(load().ks_set_option(self.h, int(option), int(value)))

    # --- states
    def set_states(self, c):
        c = np.ascontiguousarray(np.asarray(c, np.complex128).reshape(self.nstates, self.nG))
        check(load().ks_set_states(self.h, c.ctypes.data_as(ct.POINTER(ct.c_double))))

    def get_states(self, out=None):
        """The resident states as [nstates][nG] complex128; out (optional, e.g. a pinned
        buffer) receives them in place."""
        c = np.zeros((self.nstates, self.nG), np.complex128) if out is None else out
        if c.dtype != np.complex128 or c.shape != (self.nstates, self.nG) or not c.flags.c_contiguous:
            raise ValueError("out must be a contiguous [nstates][nG] complex128 array")
        check(load().ks_get_states(self.h, c.ctypes.data_as(ct.POINTER(ct.c_double))))
        return c

    def states_device_ptr(self):
        p = ct.c_void_p()
        check(load().ks_states_device(self.h, ct.byref(p)))
        return p.value

    # --- operations
    def apply_h(self, psi_ptr, hpsi_ptr, nstates, stream=None):
        check(load().ks_apply_h(self.h, ct.c_void_p(psi_ptr), ct.c_void_p(hpsi_ptr), int(nstates),
                                _stream_ptr(stream)))

    def apply_h_host(self, c):
        c = np.ascontiguousarray(np.asarray(c, np.complex128))
        out = np.zeros_like(c)
        check(load().ks_apply_h_host(self.h, c.ctypes.data_as(ct.POINTER(ct.c_double)),
                                     out.ctypes.data_as(ct.POINTER(ct.c_double)), c.shape[0]))
        return out

    def density(self, n_ptr, stream=None):
        check(load().ks_density(self.h, ct.c_void_p(n_ptr), _stream_ptr(stream)))

    def orthonormalize(self, want_S=False, stream=None):
        S = np.zeros((self.nstates, self.nstates), np.complex128) if want_S else None
        check(load().ks_orthonormalize(self.h, S.ctypes.data_as(ct.POINTER(ct.c_double)) if want_S else None,
                                       _stream_ptr(stream)))
        return S

    def rayleigh_ritz(self, stream=None):
        e = np.zeros(self.nstates)
        check(load().ks_rayleigh_ritz(self.h, _dptr(e), _stream_ptr(stream)))
        return e

    def block_iteration(self, niter, stream=None, precond=None):
        """niter block iterations; precond "teter" selects the Teter-preconditioned steepest
        descent.  Returns the Ritz values of the last iteration."""
        e = np.zeros(self.nstates)
        if precond is None:
            check(load().ks_block_iteration(self.h, int(niter), _dptr(e), _stream_ptr(stream)))
        else:
            mode = {"none": 0, "teter": 1}[precond]
            check(load().ks_block_iteration_pc(self.h, int(niter), mode, _dptr(e), _stream_ptr(stream)))
        return e

    def scf(self, max_iter, eig_iters=2, mix=0.3, tol=0.0, stream=None, mixer="linear", history=4):
        """Self-consistent field with linear, Pulay or Broyden mixing: returns (Ritz values
        [iters][nstates], density residuals [iters]) of the iterations run."""
        eig = np.zeros((max(max_iter, 1), self.nstates))
        res = np.zeros(max(max_iter, 1))
        done = ct.c_int(0)
        mode = {"linear": 0, "pulay": 1, "broyden": 2}[mixer] if isinstance(mixer, str) else int(mixer)
        check(load().ks_scf(self.h, int(max_iter), int(eig_iters), mode, float(mix), int(history), float(tol),
                            _dptr(eig), _dptr(res), ct.byref(done), _stream_ptr(stream)))
        return eig[:done.value], res[:done.value]

    def profile(self, mode):
        check(load().ks_profile(self.h, int(mode)))

    def profile_entries(self):
        """{stage name: (total ms, count)} of the accumulated stage timings."""
        out = {}
        buf = ct.create_string_buffer(128)
        ms = ct.c_double()
        cnt = ct.c_long()
        i = 0
        while load().ks_profile_read(self.h, i, buf, 128, ct.byref(ms), ct.byref(cnt)) == KS_OK:
            out[buf.value.decode()] = (ms.value, cnt.value)
            i += 1
        return out

    def profile_spans(self):
        """[(stage name, start ms, end ms)] of the timeline started by profile(3)."""
        out = []
        buf = ct.create_string_buffer(128)
        t0 = ct.c_double()
        t1 = ct.c_double()
        i = 0
        while load().ks_profile_span(self.h, i, buf, 128, ct.byref(t0), ct.byref(t1)) == KS_OK:
            out.append((buf.value.decode(), t0.value, t1.value))
            i += 1
        return out

    def td_step(self, dt, nsteps, propagator="etrs", hartree_xc=True, stream=None, dipoles=False):
        """nsteps real-time steps; returns (norms, energies), plus the dipoles [nsteps][3] at
        the start of each step when dipoles is set."""
        norms = np.zeros(nsteps)
        energies = np.zeros(nsteps)
        prop = {"etrs": 0, "taylor": 1}[propagator] if isinstance(propagator, str) else int(propagator)
        if dipoles:
            d = np.zeros((max(nsteps, 1), 3))
            check(load().ks_td_step_dipole(self.h, float(dt), int(nsteps), prop, 1 if hartree_xc else 0,
                                           _dptr(norms), _dptr(energies), _dptr(d), _stream_ptr(stream)))
            return norms, energies, d[:nsteps]
        check(load().ks_td_step(self.h, float(dt), int(nsteps), prop, 1 if hartree_xc else 0, _dptr(norms),
                                _dptr(energies), _stream_ptr(stream)))
        return norms, energies

    def kick(self, kappa, stream=None):
        """Delta kick psi <- P_S exp(i kappa . (r - L/2)) psi of every resident state."""
        k = np.ascontiguousarray(kappa, dtype=np.float64).reshape(3)
        check(load().ks_kick(self.h, _dptr(k), _stream_ptr(stream)))

    def forces(self, stream=None):
        """Forces on the atoms (Eq. 11) from the resident states, [natoms][3] Ha/bohr."""
        natoms = self.desc.natoms
        f = np.zeros((max(natoms, 1), 3))
        check(load().ks_forces(self.h, _dptr(f), _stream_ptr(stream)))
        return f[:natoms]

    def set_positions(self, pos, stream=None):
        """Moves the atoms to pos [natoms][3] (bohr): V_loc and the projectors are rebuilt."""
        p = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1)
        if p.size != 3 * self.desc.natoms:
            raise ValueError("pos must hold natoms x 3 values")
        check(load().ks_set_positions(self.h, _dptr(p) if p.size else None, _stream_ptr(stream)))

    def positions(self):
        natoms = self.desc.natoms
        p = np.zeros((max(natoms, 1), 3))
        check(load().ks_get_positions(self.h, _dptr(p)))
        return p[:natoms]

    def ehrenfest(self, dt, nsteps, mass, vel, hartree_xc=True, stream=None):
        """Ehrenfest dynamics (ETRS electrons, velocity-Verlet ions): returns (positions
        [nsteps][natoms][3], final velocities [natoms][3], total energies [nsteps])."""
        natoms = self.desc.natoms
        m = np.ascontiguousarray(np.broadcast_to(np.asarray(mass, np.float64), (natoms,)))
        v = np.ascontiguousarray(vel, dtype=np.float64).reshape(natoms, 3).copy()
        pos = np.zeros((max(nsteps, 1), max(natoms, 1), 3))
        e = np.zeros(max(nsteps, 1))
        check(load().ks_ehrenfest(self.h, float(dt), int(nsteps), 1 if hartree_xc else 0,
                                  _dptr(m) if natoms else None, _dptr(v) if natoms else None,
                                  _dptr(pos), _dptr(e), _stream_ptr(stream)))
        return pos[:nsteps, :natoms], v, e[:nsteps]

    def dipole(self, stream=None):
        """dV sum_j (r_j - L/2) n(r_j) of the resident states."""
        d = np.zeros(3)
        check(load().ks_dipole(self.h, _dptr(d), _stream_ptr(stream)))
        return d


class Server:
    """Owns a ks_server (continuous batching of independent calculations)."""

    def __init__(self, budget_bytes=0, workers=0):
        self.h = ct.c_void_p()
        check(load().ks_serve_create_ex(ct.c_size_t(int(budget_bytes)), int(workers), ct.byref(self.h)))
        self._descs = {}

    def close(self):
        if self.h:
            load().ks_serve_destroy(self.h)
            self.h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, cell, kind, count, dt=0.05, c0=None, prec="bf16x3", nstates=None):
        """kind 0: `count` block iterations; kind 1: `count` ETRS steps (Hartree + exchange)."""
        d = make_desc(cell, prec, nstates)
        arr = None
        if c0 is not None:
            arr = np.ascontiguousarray(np.asarray(c0, np.complex128))
        t = ct.c_uint64()
        check(load().ks_serve_submit(self.h, ct.byref(d), arr.ctypes.data_as(ct.POINTER(ct.c_double))
                                     if arr is not None else None, int(kind), int(count), float(dt), ct.byref(t)))
        self._descs[t.value] = d
        return t.value

    def stats(self):
        """Worker seconds by activity and group counts since creation (ks_serve_stats)."""
        v = np.zeros(14)
        check(load().ks_serve_stats(self.h, _dptr(v), 14))
        keys = ("start_s", "ground_state_s", "realtime_s", "retire_s", "starts", "ground_state_quanta",
                "realtime_group_steps", "realtime_request_steps", "pool_bytes", "start_create_s", "start_init_s",
                "start_orthonormalize_s", "pool_slabs_allocated", "pool_alloc_s")
        return dict(zip(keys, v.tolist()))

    def poll(self, ticket, timeout_ms=0, want_states=False):
        """(status, result, states or None, latency_s); status KS_PENDING while running."""
        nres, ns, nG = ct.c_int(), ct.c_int(), ct.c_int()
        st = load().ks_serve_result_info(self.h, ct.c_uint64(ticket), ct.byref(nres), ct.byref(ns), ct.byref(nG))
        if st != KS_OK:
            return st, None, None, None
        res = np.zeros(nres.value)
        states = np.zeros((ns.value, nG.value), np.complex128) if want_states else None
        lat = ct.c_double()
        st = load().ks_serve_poll(self.h, ct.c_uint64(ticket), int(timeout_ms), _dptr(res),
                                  states.ctypes.data_as(ct.POINTER(ct.c_double)) if want_states else None,
                                  ct.byref(lat))
        if st == KS_OK:
            self._descs.pop(ticket, None)
        return st, res, states, lat.value
