"""ctypes binding of the C ABI in include/lowmach.h (same names, argument
marshalling only -- every step of the method runs in the CUDA library).

PyTorch supplies the device memory (one workspace tensor per simulation) and
the CUDA stream; nothing here computes on the CPU.  Loading fails loudly when
the shared library has not been built.
"""

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblowmach.so")

SIM_OK, SIM_EINVAL, SIM_ENOMEM, SIM_ECUDA, SIM_ENOCONV, SIM_ENAN, SIM_EUNSTABLE, SIM_ESTATE = \
    0, -1, -2, -3, -4, -5, -6, -7
STATUS_NAMES = {0: "SIM_OK", -1: "SIM_EINVAL", -2: "SIM_ENOMEM", -3: "SIM_ECUDA", -4: "SIM_ENOCONV",
                -5: "SIM_ENAN", -6: "SIM_EUNSTABLE", -7: "SIM_ESTATE"}
SIM_BC_PERIODIC, SIM_BC_INFLOW, SIM_BC_OUTFLOW, SIM_BC_WALL, SIM_BC_SLIP, SIM_BC_WALL_T = 0, 1, 2, 3, 4, 5
SIM_FP64, SIM_MIXED = 0, 1
SIM_IBM_NONE, SIM_IBM_SLOT, SIM_IBM_SPHERE, SIM_IBM_MARKERS, SIM_IBM_COUETTE = 0, 1, 2, 3, 4
(SIM_FIELD_U, SIM_FIELD_V, SIM_FIELD_W, SIM_FIELD_Z, SIM_FIELD_H, SIM_FIELD_T, SIM_FIELD_RHO,
 SIM_FIELD_P, SIM_FIELD_FX, SIM_FIELD_FY, SIM_FIELD_FZ, SIM_FIELD_CHI, SIM_FIELD_SM,
 SIM_FIELD_KAPPA) = range(14)
SIM_GET, SIM_SET = 0, 1
(SIM_K_RESIDUAL, SIM_K_MG_DOWN, SIM_K_CG_MATVEC, SIM_K_MG_UP, SIM_K_STATE, SIM_K_PROJECT,
 SIM_K_MG_TAIL, SIM_K_RESIDUAL_REV) = range(8)
(SIM_Q_TIME, SIM_Q_DT, SIM_Q_P0, SIM_Q_STEPS, SIM_Q_ITERS_PRED, SIM_Q_ITERS_CORR, SIM_Q_RESID_PRED,
 SIM_Q_RESID_CORR, SIM_Q_MASS, SIM_Q_NCELLS, SIM_Q_MG_LEVELS, SIM_Q_KERNEL_LAUNCHES, SIM_Q_TAIL_NX,
 SIM_Q_TAIL_NY, SIM_Q_TAIL_FDM, SIM_Q_TAIL_NZ, SIM_Q_DIV_RESID, SIM_Q_DIV_SCALE, SIM_Q_MASS_BALANCE,
 SIM_Q_PC_DIFF_U, SIM_Q_PC_DIFF_V, SIM_Q_PC_DIFF_W, SIM_Q_PC_DIFF_P) = range(23)

FIELD_IDS = dict(U=SIM_FIELD_U, V=SIM_FIELD_V, W=SIM_FIELD_W, Z=SIM_FIELD_Z, H=SIM_FIELD_H,
                 T=SIM_FIELD_T, RHO=SIM_FIELD_RHO, P=SIM_FIELD_P, FX=SIM_FIELD_FX, FY=SIM_FIELD_FY,
                 FZ=SIM_FIELD_FZ, CHI=SIM_FIELD_CHI, SM=SIM_FIELD_SM, KAPPA=SIM_FIELD_KAPPA)


class SimParams(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("L", ctypes.c_double * 3),
                ("bc", (ctypes.c_int * 2) * 3), ("inflow_v", ctypes.c_double * 3),
                ("inflow_Z", ctypes.c_double), ("inflow_H", ctypes.c_double),
                ("Re", ctypes.c_double), ("Pr", ctypes.c_double), ("inv_Fr2", ctypes.c_double),
                ("Le_F", ctypes.c_double), ("Le_O", ctypes.c_double), ("gamma", ctypes.c_double),
                ("sigma", ctypes.c_double), ("transport", ctypes.c_int),
                ("sutherland_C", ctypes.c_double), ("wall_H", (ctypes.c_double * 2) * 3),
                ("Z_st", ctypes.c_double),
                ("density_ratio", ctypes.c_double), ("eps_reg", ctypes.c_double),
                ("tol_reg", ctypes.c_double), ("closed_system", ctypes.c_int),
                ("incompressible", ctypes.c_int), ("dt", ctypes.c_double),
                ("precision", ctypes.c_int), ("poisson_rtol", ctypes.c_double),
                ("poisson_max_iter", ctypes.c_int), ("mg_sweeps", ctypes.c_int),
                ("mg_tail_cells", ctypes.c_int), ("stage_tile_x", ctypes.c_int)]


class SimIbm(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("center", ctypes.c_double * 3), ("half", ctypes.c_double * 3),
                ("radius", ctypes.c_double), ("Da_ib", ctypes.c_double), ("rho_b", ctypes.c_double),
                ("U_b", ctypes.c_double), ("Z_ib", ctypes.c_double), ("H_ib", ctypes.c_double),
                ("n_profile", ctypes.c_int), ("profile", ctypes.POINTER(ctypes.c_double)),
                ("n_markers", ctypes.c_int), ("markers", ctypes.POINTER(ctypes.c_double))]


_lib = None


def load():
    """The loaded shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run paper_2603_01727_gb300.build)")
    lib = ctypes.CDLL(LIB_PATH)
    P, VP, I, D, SZ = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sig = {
        "sim_workspace_size": ([P(SimParams), P(SZ)], I),
        "sim_create": ([P(SimParams), VP, SZ, VP, P(VP)], I),
        "sim_set_ibm_geometry": ([VP, P(SimIbm)], I),
        "sim_fields": ([VP, I, VP, I, I], I),
        "sim_step": ([VP, I], I),
        "sim_sync": ([VP], I),
        "sim_query": ([VP, I, P(D)], I),
        "sim_last_error": ([VP], ctypes.c_char_p),
        "sim_destroy": ([VP], None),
        "sim_time_kernel": ([VP, I, I], I),
        "sim_state_size": ([VP, P(SZ)], I),
        "sim_state_save": ([VP, VP, I], I),
        "sim_state_load": ([VP, VP, I], I),
        "sim_step_save": ([VP, VP, I], I),
        "sim_poisson_workspace_size": ([I, P(I), P(I), P(SZ)], I),
        "sim_poisson_solve": ([I, P(I), P(D), P(I), VP, VP, D, I, VP, SZ, VP, P(I), P(D)], I),
        "sim_poisson_solve_noalloc": ([I, P(I), P(D), P(I), VP, VP, D, I, VP, P(I), P(D)], I),
        "sim_poisson_batch_workspace_size": ([P(I), P(I), I, I, P(SZ)], I),
        "sim_poisson_solve_batch": ([P(I), P(D), P(I), I, I, VP, VP, D, I, VP, SZ, VP, P(I), P(D)], I),
        "sim_objective": ([VP, P(D)], I),
        "sim_adjoint_workspace_size": ([VP, P(SZ)], I),
        "sim_adjoint_begin": ([VP, VP, SZ], I),
        "sim_adjoint_step": ([VP, D, P(D)], I),
        "sim_adjoint_field": ([VP, I, VP, I], I),
        "sim_adjoint_end": ([VP], I),
        "sim_batch_workspace_size": ([P(VP), I, P(SZ)], I),
        "sim_batch_create": ([P(VP), I, VP, SZ, VP, P(VP)], I),
        "sim_batch_query_launches": ([VP, P(D)], I),
        "sim_batch_step": ([VP, I], I),
        "sim_batch_sync": ([VP], I),
        "sim_batch_last_error": ([VP], ctypes.c_char_p),
        "sim_batch_destroy": ([VP], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def exported_symbols():
    return ["sim_workspace_size", "sim_create", "sim_set_ibm_geometry", "sim_fields", "sim_step",
            "sim_sync", "sim_query", "sim_last_error", "sim_destroy", "sim_time_kernel", "sim_state_size",
            "sim_state_save",
            "sim_state_load", "sim_step_save", "sim_poisson_workspace_size",
            "sim_poisson_solve", "sim_poisson_solve_noalloc", "sim_poisson_batch_workspace_size",
            "sim_poisson_solve_batch", "sim_objective", "sim_adjoint_workspace_size",
            "sim_adjoint_begin", "sim_adjoint_step", "sim_adjoint_field", "sim_adjoint_end",
            "sim_batch_workspace_size", "sim_batch_create", "sim_batch_query_launches", "sim_batch_step",
            "sim_batch_sync", "sim_batch_last_error", "sim_batch_destroy"]


class SimError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def params_struct(prm):
    if any(float(a) != 0.0 for a in prm.get("stretch", [])):
        # the kernels read one spacing per direction
        raise ValueError("stretched grids (Eq 4.18) are not supported by the CUDA path")
    p = SimParams()
    p.dim = int(prm["dim"])
    for d in range(3):
        p.n[d] = int(prm["n"][d])
        p.L[d] = float(prm["L"][d])
        p.inflow_v[d] = float(prm["inflow_v"][d])
        for s in range(2):
            p.bc[d][s] = int(prm["bc"][d][s])
    for k in ("inflow_Z", "inflow_H", "Re", "Pr", "inv_Fr2", "Le_F", "Le_O", "gamma", "sigma", "Z_st",
              "density_ratio", "eps_reg", "tol_reg", "dt", "poisson_rtol"):
        setattr(p, k, float(prm[k]))
    for k in ("closed_system", "incompressible", "precision", "poisson_max_iter"):
        setattr(p, k, int(prm[k]))
    p.mg_sweeps = int(prm.get("mg_sweeps", 0))
    p.mg_tail_cells = int(prm.get("mg_tail_cells", 0))
    p.stage_tile_x = int(prm.get("stage_tile_x", 0))
    p.transport = int(prm.get("transport", 0))
    p.sutherland_C = float(prm.get("sutherland_C", 0.0))
    wall_H = prm.get("wall_H")
    for d in range(3):
        for s in range(2):
            p.wall_H[d][s] = float(wall_H[d][s]) if wall_H is not None and d < len(wall_H) else 0.0
    return p


def ibm_struct(geo):
    b = SimIbm()
    if geo is None:
        b.kind = SIM_IBM_NONE
        return b, None
    b.kind = int(geo["kind"])
    for d in range(3):
        b.center[d] = float(geo["center"][d]) if d < len(geo["center"]) else 0.0
        half = geo.get("half", [0.0, 0.0, 0.0])
        b.half[d] = float(half[d]) if d < len(half) else 0.0
    b.radius = float(geo.get("radius", 0.0))
    for k in ("Da_ib", "rho_b", "U_b", "Z_ib", "H_ib"):
        setattr(b, k, float(geo[k]))
    prof = geo.get("profile")
    keep = []
    if prof is not None and len(prof) > 0:
        arr = np.ascontiguousarray(np.asarray(prof, dtype=np.float64))
        keep.append(arr)
        b.n_profile = len(arr)
        b.profile = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    mk = geo.get("markers")
    if mk is not None and len(mk) > 0:
        arr = np.ascontiguousarray(np.asarray(mk, dtype=np.float64))
        keep.append(arr)
        b.n_markers = arr.shape[0]
        b.markers = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return b, keep


def _check(lib, st, handle=None):
    if st != SIM_OK:
        msg = lib.sim_last_error(handle).decode() if handle else ""
        raise SimError(st, msg)


class Simulation:
    """Thin owner of one sim_t: the torch workspace tensor, the handle and the stream."""

    def __init__(self, prm, geo=None, device="cuda", stream=None):
        import torch
        self.lib = load()
        self.torch = torch
        self.prm = dict(prm)
        self._p = params_struct(prm)
        sz = ctypes.c_size_t()
        _check(self.lib, self.lib.sim_workspace_size(ctypes.byref(self._p), ctypes.byref(sz)))
        self.workspace_bytes = sz.value
        self.workspace = torch.empty(sz.value + 256, dtype=torch.uint8, device=device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = ctypes.c_void_p()
        _check(self.lib, self.lib.sim_create(ctypes.byref(self._p), ctypes.c_void_p(self._ws_ptr),
                                             ctypes.c_size_t(sz.value),
                                             ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h
        self.dim = int(prm["dim"])
        self.n = [int(v) for v in prm["n"][: self.dim]]
        self.set_ibm(geo)

    def set_ibm(self, geo):
        b, keep = ibm_struct(geo)
        _check(self.lib, self.lib.sim_set_ibm_geometry(self.h, ctypes.byref(b)), self.h)
        del keep

    def shape(self, face_dir=None):
        m = list(self.n)
        if face_dir is not None:
            m[face_dir] += 1
        return tuple(reversed(m))

    def set_field(self, name, arr):
        """Copy an interior array (numpy on the host, or a CUDA torch tensor) in."""
        fid = FIELD_IDS[name]
        if isinstance(arr, np.ndarray):
            a = np.ascontiguousarray(arr, dtype=np.float64)
            assert a.shape == self.shape(), (a.shape, self.shape())
            _check(self.lib, self.lib.sim_fields(self.h, fid, a.ctypes.data_as(ctypes.c_void_p), SIM_SET, 0),
                   self.h)
        else:
            t = arr.contiguous()
            assert t.dtype == self.torch.float64 and t.is_cuda
            _check(self.lib, self.lib.sim_fields(self.h, fid, ctypes.c_void_p(t.data_ptr()), SIM_SET, 1),
                   self.h)

    def set_fields(self, fields):
        for d in range(self.dim):
            self.set_field("UVW"[d], fields["v"][d])
        self.set_field("Z", fields["Z"])
        self.set_field("H", fields["H"])

    def get(self, name, out=None):
        """Copy a field out: a new numpy array, or into the given CUDA tensor."""
        fid = FIELD_IDS[name]
        face = {"FX": 0, "FY": 1, "FZ": 2}.get(name)
        if out is None:
            a = np.empty(self.shape(face), dtype=np.float64)
            _check(self.lib, self.lib.sim_fields(self.h, fid, a.ctypes.data_as(ctypes.c_void_p), SIM_GET, 0),
                   self.h)
            return a
        _check(self.lib, self.lib.sim_fields(self.h, fid, ctypes.c_void_p(out.data_ptr()), SIM_GET, 1), self.h)
        return out

    def step(self, nsteps=1):
        _check(self.lib, self.lib.sim_step(self.h, int(nsteps)), self.h)

    def sync(self):
        _check(self.lib, self.lib.sim_sync(self.h), self.h)

    def query(self, what):
        v = ctypes.c_double()
        _check(self.lib, self.lib.sim_query(self.h, int(what), ctypes.byref(v)), self.h)
        return v.value

    def time_kernel(self, kernel, reps):
        """Enqueue reps launches of one step kernel (SIM_K_*) on the stream."""
        _check(self.lib, self.lib.sim_time_kernel(self.h, int(kernel), int(reps)), self.h)

    def state_size(self):
        sz = ctypes.c_size_t()
        _check(self.lib, self.lib.sim_state_size(self.h, ctypes.byref(sz)), self.h)
        return sz.value

    def state_save(self, buf):
        """Copy the restart state into a uint8 buffer (numpy or CUDA/pinned torch tensor)."""
        ptr, dev = self._buf(buf)
        _check(self.lib, self.lib.sim_state_save(self.h, ptr, dev), self.h)

    def state_load(self, buf):
        ptr, dev = self._buf(buf)
        _check(self.lib, self.lib.sim_state_load(self.h, ptr, dev), self.h)

    def step_save(self, buf):
        """One step, its restart blob copied into buf while the step runs."""
        ptr, dev = self._buf(buf)
        _check(self.lib, self.lib.sim_step_save(self.h, ptr, dev), self.h)

    # --------------------------- objective and adjoint ---------------------------
    def objective(self):
        """Heat-release integral sum(omega dV) at the current level (synchronous)."""
        v = ctypes.c_double()
        _check(self.lib, self.lib.sim_objective(self.h, ctypes.byref(v)), self.h)
        return v.value

    def adjoint_begin(self):
        """Allocate the adjoint workspace and zero the adjoint state."""
        sz = ctypes.c_size_t()
        _check(self.lib, self.lib.sim_adjoint_workspace_size(self.h, ctypes.byref(sz)), self.h)
        self._adj_ws = self.torch.empty(sz.value + 256, dtype=self.torch.uint8, device=self.workspace.device)
        ptr = (self._adj_ws.data_ptr() + 255) // 256 * 256
        _check(self.lib, self.lib.sim_adjoint_begin(self.h, ctypes.c_void_p(ptr), ctypes.c_size_t(sz.value)),
               self.h)

    def adjoint_step(self, objective_weight=0.0, n_profile=0):
        """Recompute the step from the loaded level n and transpose it; with
        n_profile > 0, also return the gradient with respect to the profile
        samples accumulated so far (numpy)."""
        if n_profile > 0:
            g = np.zeros(int(n_profile), dtype=np.float64)
            ptr = g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        else:
            g, ptr = None, None
        _check(self.lib, self.lib.sim_adjoint_step(self.h, float(objective_weight), ptr), self.h)
        return g

    def adjoint_get(self, name):
        fid = FIELD_IDS[name]
        face = {"FX": 0, "FY": 1, "FZ": 2}.get(name)
        a = np.empty(self.shape(face), dtype=np.float64)
        _check(self.lib, self.lib.sim_adjoint_field(self.h, fid, a.ctypes.data_as(ctypes.c_void_p), SIM_GET),
               self.h)
        return a

    def adjoint_seed(self, name, arr):
        """Add arr (interior cells) to the adjoint of a state field."""
        a = np.ascontiguousarray(arr, dtype=np.float64)
        assert a.shape == self.shape()
        _check(self.lib, self.lib.sim_adjoint_field(self.h, FIELD_IDS[name], a.ctypes.data_as(ctypes.c_void_p),
                                                    SIM_SET), self.h)

    def adjoint_end(self):
        _check(self.lib, self.lib.sim_adjoint_end(self.h), self.h)
        self._adj_ws = None

    def _buf(self, buf):
        if isinstance(buf, np.ndarray):
            return buf.ctypes.data_as(ctypes.c_void_p), 0
        return ctypes.c_void_p(buf.data_ptr()), int(buf.is_cuda)

    def close(self):
        if getattr(self, "h", None):
            self.lib.sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def poisson_solve(b, P, h, periodic, rtol=1e-12, max_iter=200, stream=None):
    """Stand-alone pressure solve on CUDA float64 tensors b, P (interior shape,
    x fastest); P holds the warm start and receives the zero-mean solution.
    Returns (iterations, final relative residual)."""
    import torch
    lib = load()
    dim = b.dim()
    n = (ctypes.c_int * 3)(*([int(s) for s in reversed(b.shape)] + [1] * (3 - dim)))
    per = (ctypes.c_int * 3)(*([int(bool(x)) for x in periodic] + [0] * (3 - dim)))
    hh = (ctypes.c_double * 3)(*([float(x) for x in h] + [1.0] * (3 - dim)))
    sz = ctypes.c_size_t()
    _check(lib, lib.sim_poisson_workspace_size(dim, n, per, ctypes.byref(sz)))
    ws = torch.empty(sz.value + 256, dtype=torch.uint8, device=b.device)
    ptr = (ws.data_ptr() + 255) // 256 * 256
    st = stream if stream is not None else torch.cuda.current_stream(b.device)
    it = ctypes.c_int()
    rr = ctypes.c_double()
    status = lib.sim_poisson_solve(dim, n, hh, per, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(P.data_ptr()),
                                   float(rtol), int(max_iter), ctypes.c_void_p(ptr), ctypes.c_size_t(sz.value),
                                   ctypes.c_void_p(st.cuda_stream), ctypes.byref(it), ctypes.byref(rr))
    _check(lib, status)
    return it.value, rr.value


def poisson_solve_batch(b, P, h, periodic, precision=SIM_FP64, rtol=1e-12, max_iter=200, stream=None):
    """Batched stand-alone pressure solve: b, P CUDA float64 tensors of shape
    (nb, n1, n0), nb independent 2D systems on one grid, advanced together.
    Returns (iterations per system, final relative residual per system)."""
    import torch
    lib = load()
    assert b.dim() == 3 and b.shape == P.shape
    nb = int(b.shape[0])
    n = (ctypes.c_int * 2)(int(b.shape[2]), int(b.shape[1]))
    per = (ctypes.c_int * 2)(*[int(bool(x)) for x in periodic])
    hh = (ctypes.c_double * 2)(*[float(x) for x in h])
    sz = ctypes.c_size_t()
    _check(lib, lib.sim_poisson_batch_workspace_size(n, per, nb, int(precision), ctypes.byref(sz)))
    ws = torch.empty(sz.value + 256, dtype=torch.uint8, device=b.device)
    ptr = (ws.data_ptr() + 255) // 256 * 256
    st = stream if stream is not None else torch.cuda.current_stream(b.device)
    it = (ctypes.c_int * nb)()
    rr = (ctypes.c_double * nb)()
    status = lib.sim_poisson_solve_batch(n, hh, per, nb, int(precision), ctypes.c_void_p(b.data_ptr()),
                                         ctypes.c_void_p(P.data_ptr()), float(rtol), int(max_iter),
                                         ctypes.c_void_p(ptr), ctypes.c_size_t(sz.value),
                                         ctypes.c_void_p(st.cuda_stream), it, rr)
    _check(lib, status)
    return list(it), list(rr)


def poisson_solve_noalloc(b, P, h, periodic, rtol=1e-12, max_iter=200, stream=None):
    """Same as poisson_solve, through sim_poisson_solve_noalloc: the library
    uses its own static device scratch, so nothing is allocated for the call
    (the caller still owns b and P).  Returns (iterations, relative residual)."""
    import torch
    lib = load()
    dim = b.dim()
    n = (ctypes.c_int * 3)(*([int(s) for s in reversed(b.shape)] + [1] * (3 - dim)))
    per = (ctypes.c_int * 3)(*([int(bool(x)) for x in periodic] + [0] * (3 - dim)))
    hh = (ctypes.c_double * 3)(*([float(x) for x in h] + [1.0] * (3 - dim)))
    st = stream if stream is not None else torch.cuda.current_stream(b.device)
    it = ctypes.c_int()
    rr = ctypes.c_double()
    status = lib.sim_poisson_solve_noalloc(dim, n, hh, per, ctypes.c_void_p(b.data_ptr()),
                                           ctypes.c_void_p(P.data_ptr()), float(rtol), int(max_iter),
                                           ctypes.c_void_p(st.cuda_stream), ctypes.byref(it), ctypes.byref(rr))
    _check(lib, status)
    return it.value, rr.value


class Batch:
    """Independent simulations advanced together, one CUDA graph per step
    (sim_batch_* of the C ABI).  The Simulation objects stay owned by the
    caller and must outlive the batch."""

    def __init__(self, sims, stream=None, batched_solves=True):
        """batched_solves: same-grid members share one batched pressure solve
        per stage (a torch workspace is allocated for it); False keeps every
        member's own solves."""
        import torch
        self.lib = load()
        self.sims = list(sims)
        arr = (ctypes.c_void_p * len(self.sims))(*[s.h.value for s in self.sims])
        st = stream if stream is not None else self.sims[0].stream
        self.stream = st
        self.workspace = None
        ptr, nbytes = None, 0
        if batched_solves:
            sz = ctypes.c_size_t()
            _check(self.lib, self.lib.sim_batch_workspace_size(arr, len(self.sims), ctypes.byref(sz)))
            if sz.value > 0:
                self.workspace = torch.empty(sz.value + 256, dtype=torch.uint8, device=self.sims[0].workspace.device)
                ptr = (self.workspace.data_ptr() + 255) // 256 * 256
                nbytes = sz.value
        h = ctypes.c_void_p()
        _check(self.lib, self.lib.sim_batch_create(arr, len(self.sims), ctypes.c_void_p(ptr), ctypes.c_size_t(nbytes),
                                                   ctypes.c_void_p(st.cuda_stream), ctypes.byref(h)))
        self.h = h
        self.torch = torch

    def launches(self):
        """Kernels launched by the last batch step (synchronises)."""
        v = ctypes.c_double()
        self._check(self.lib.sim_batch_query_launches(self.h, ctypes.byref(v)))
        return v.value

    def _check(self, st):
        if st != SIM_OK:
            raise SimError(st, self.lib.sim_batch_last_error(self.h).decode())

    def step(self, nsteps=1):
        self._check(self.lib.sim_batch_step(self.h, int(nsteps)))

    def sync(self):
        self._check(self.lib.sim_batch_sync(self.h))

    def cells(self):
        return sum(int(s.query(SIM_Q_NCELLS)) for s in self.sims)

    def close(self):
        if getattr(self, "h", None):
            self.lib.sim_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
