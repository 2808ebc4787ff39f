"""Thin ctypes binding of libaccfem.so (include/accfem.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; there is no Python or CPU fallback.
Loading fails loudly when the library has not been built.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libaccfem.so")

OK, E_INVALID_ARG, E_NOMEM, E_CUDA, E_NOT_CONVERGED, E_CONTACT_CAPACITY, E_NOT_SPD, E_TIMEOUT, E_PENETRATION = range(9)

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


class accfem_robot_desc(ctypes.Structure):
    _fields_ = [("length", ctypes.c_double), ("outer_radius", ctypes.c_double), ("inner_radius", ctypes.c_double),
                ("youngs_modulus", ctypes.c_double), ("poisson_ratio", ctypes.c_double),
                ("n_elements", ctypes.c_int32), ("n_cables", ctypes.c_int32), ("cable_radius", ctypes.c_double),
                ("cable_angles", _dp)]


class accfem_lumen_desc(ctypes.Structure):
    _fields_ = [("vertices", _dp), ("n_vertices", ctypes.c_int64), ("triangles", _ip), ("n_triangles", ctypes.c_int64),
                ("entrance_point", ctypes.c_double * 3), ("entrance_dir", ctypes.c_double * 3),
                ("entrance_up", ctypes.c_double * 3)]


class accfem_options(ctypes.Structure):
    _fields_ = [("activation_gap", ctypes.c_double), ("step_limit", ctypes.c_double), ("newton_tol", ctypes.c_double),
                ("contact_tol", ctypes.c_double), ("max_newton_iters", ctypes.c_int32),
                ("max_contact_iters", ctypes.c_int32), ("max_contacts", ctypes.c_int32),
                ("tangent_mode", ctypes.c_int32)]


class accfem_result(ctypes.Structure):
    _fields_ = [("node_pos", _dp), ("node_quat", _dp), ("contact_capacity", ctypes.c_int32),
                ("n_contacts", ctypes.c_int32), ("contact_node", _ip), ("contact_tri", _ip),
                ("contact_point", _dp), ("contact_normal", _dp), ("contact_force", _dp),
                ("base_reaction", ctypes.c_double * 6), ("newton_iters", ctypes.c_int32),
                ("contact_iters", ctypes.c_int32), ("residual", ctypes.c_double)]


class accfem_request(ctypes.Structure):
    _fields_ = [("arrival", ctypes.c_double), ("member", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("cable_tensions", ctypes.c_double * 8), ("insertion", ctypes.c_double)]


class accfem_response(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("newton_iters", ctypes.c_int32), ("t_begin", ctypes.c_double),
                ("t_end", ctypes.c_double), ("tip", ctypes.c_double * 7), ("n_contacts", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


REQUEST_DTYPE = np.dtype([("arrival", np.float64), ("member", np.int32), ("pad", np.int32),
                          ("cable_tensions", np.float64, (8,)), ("insertion", np.float64)], align=True)
RESPONSE_DTYPE = np.dtype([("status", np.int32), ("newton_iters", np.int32), ("t_begin", np.float64),
                           ("t_end", np.float64), ("tip", np.float64, (7,)), ("n_contacts", np.int32),
                           ("pad", np.int32)], align=True)
assert REQUEST_DTYPE.itemsize == ctypes.sizeof(accfem_request)
assert RESPONSE_DTYPE.itemsize == ctypes.sizeof(accfem_response)


class accfem_state(ctypes.Structure):
    _fields_ = [("node_pos", _dp), ("node_quat", _dp)]


EXPORTS = ["accfem_default_options", "accfem_create", "accfem_solve", "accfem_solve_tip_load",
           "accfem_solve_resident", "accfem_reset", "accfem_set_stream", "accfem_transfer_bytes",
           "accfem_time_kernel", "accfem_time_kernel_graph", "accfem_get_state", "accfem_kernel_launches",
           "accfem_destroy",
           "accfem_status_string", "accfem_last_error", "accfem_detect_contacts_noalloc",
           "accfem_batch_create", "accfem_batch_begin", "accfem_batch_advance", "accfem_batch_poll",
           "accfem_batch_results", "accfem_batch_solve", "accfem_batch_set_stream", "accfem_batch_transfer_bytes",
           "accfem_batch_kernel_launches", "accfem_batch_last_error", "accfem_batch_destroy", "accfem_batch_serve",
           "accfem_device_bytes", "accfem_solve_stats", "accfem_solve_admm_iterations", "accfem_set_precision",
           "accfem_batch_autotune",
           "accfem_batch_tuning", "accfem_set_element_modulus", "accfem_set_frame_mode",
           "accfem_set_contact_solver", "accfem_batch_time_phase", "accfem_set_contact_model"]

PRECISION_FP64, PRECISION_MIXED = 0, 1
CONTACT_ACTIVE_SET, CONTACT_ADMM, CONTACT_PRIMAL_ADMM = 0, 1, 2
CONTACT_NODE, CONTACT_SEGMENT = 0, 1

MAX_CABLES = 8

KERNEL_ELEMENT, KERNEL_COLLIDE, KERNEL_ASSEMBLE, KERNEL_CONTACT, KERNEL_FACTOR = range(5)

_lib = None


def load(path=LIB_PATH):
    """Loads libaccfem.so and declares the C signatures; raises if the library is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libaccfem.so not built (%s); run paper_2503_06922_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    H = ctypes.c_void_p
    lib.accfem_default_options.argtypes = [ctypes.POINTER(accfem_options)]
    lib.accfem_create.argtypes = [ctypes.POINTER(accfem_robot_desc), ctypes.POINTER(accfem_lumen_desc),
                                  ctypes.POINTER(accfem_options), ctypes.POINTER(H)]
    lib.accfem_solve.argtypes = [H, _dp, ctypes.c_double, ctypes.POINTER(accfem_state), ctypes.POINTER(accfem_result)]
    lib.accfem_solve_tip_load.argtypes = [H, _dp, _dp, ctypes.c_int32, ctypes.c_double, ctypes.POINTER(accfem_state),
                                          ctypes.POINTER(accfem_result)]
    lib.accfem_solve_resident.argtypes = [H, ctypes.c_void_p, ctypes.c_double, _ip]
    lib.accfem_get_state.argtypes = [H, _dp, _dp]
    lib.accfem_reset.argtypes = [H]
    lib.accfem_set_stream.argtypes = [H, ctypes.c_void_p]
    lib.accfem_transfer_bytes.argtypes = [H, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.accfem_time_kernel.argtypes = [H, ctypes.c_int, ctypes.c_int32, _dp]
    lib.accfem_time_kernel_graph.argtypes = [H, ctypes.c_int, ctypes.c_int32, _dp]
    lib.accfem_detect_contacts_noalloc.argtypes = [H, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.c_void_p, ctypes.c_void_p]
    lib.accfem_kernel_launches.argtypes = [H]
    lib.accfem_kernel_launches.restype = ctypes.c_int64
    lib.accfem_destroy.argtypes = [H]
    lib.accfem_destroy.restype = None
    lib.accfem_status_string.argtypes = [ctypes.c_int]
    lib.accfem_status_string.restype = ctypes.c_char_p
    lib.accfem_last_error.argtypes = [H]
    lib.accfem_last_error.restype = ctypes.c_char_p
    B = ctypes.c_void_p
    lib.accfem_batch_create.argtypes = [ctypes.POINTER(H), ctypes.c_int32, ctypes.POINTER(B)]
    lib.accfem_batch_begin.argtypes = [B, ctypes.c_int32, _dp, ctypes.c_double]
    lib.accfem_batch_advance.argtypes = [B, ctypes.c_int32, _ip]
    lib.accfem_batch_poll.argtypes = [B, ctypes.c_int32, _ip, ctypes.POINTER(ctypes.c_int), _ip]
    lib.accfem_batch_results.argtypes = [B, _ip, ctypes.c_int32, ctypes.POINTER(accfem_result),
                                         ctypes.POINTER(ctypes.c_int)]
    lib.accfem_batch_solve.argtypes = [B, _dp, _dp, _ip, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(accfem_result)]
    lib.accfem_batch_set_stream.argtypes = [B, ctypes.c_void_p]
    lib.accfem_batch_transfer_bytes.argtypes = [B, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.accfem_batch_kernel_launches.argtypes = [B]
    lib.accfem_batch_kernel_launches.restype = ctypes.c_int64
    lib.accfem_batch_last_error.argtypes = [B]
    lib.accfem_batch_last_error.restype = ctypes.c_char_p
    lib.accfem_batch_serve.argtypes = [B, ctypes.POINTER(accfem_request), ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int64, ctypes.POINTER(accfem_response), ctypes.POINTER(accfem_result)]
    lib.accfem_device_bytes.argtypes = [H, ctypes.POINTER(ctypes.c_int64)]
    lib.accfem_solve_stats.argtypes = [H, _ip, _ip, _ip, _ip]
    lib.accfem_solve_admm_iterations.argtypes = [H, _ip]
    lib.accfem_set_precision.argtypes = [H, ctypes.c_int32]
    lib.accfem_set_element_modulus.argtypes = [H, _dp, ctypes.c_int32]
    lib.accfem_set_frame_mode.argtypes = [H, ctypes.c_int32]
    lib.accfem_set_contact_solver.argtypes = [H, ctypes.c_int32]
    lib.accfem_set_contact_model.argtypes = [H, ctypes.c_int32]
    lib.accfem_batch_autotune.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    lib.accfem_batch_tuning.argtypes = [ctypes.c_void_p, _ip, _dp]
    lib.accfem_batch_time_phase.argtypes = [B, ctypes.c_int, ctypes.c_int32, _dp, ctypes.POINTER(ctypes.c_int64)]
    lib.accfem_batch_destroy.argtypes = [B]
    lib.accfem_batch_destroy.restype = None
    for name in ("accfem_default_options", "accfem_create", "accfem_solve", "accfem_solve_tip_load",
                 "accfem_solve_resident", "accfem_get_state", "accfem_reset", "accfem_set_stream",
                 "accfem_transfer_bytes", "accfem_time_kernel", "accfem_time_kernel_graph",
                 "accfem_detect_contacts_noalloc",
                 "accfem_batch_create", "accfem_batch_begin", "accfem_batch_advance", "accfem_batch_poll",
                 "accfem_batch_results", "accfem_batch_solve", "accfem_batch_set_stream",
                 "accfem_batch_transfer_bytes", "accfem_batch_serve", "accfem_device_bytes", "accfem_solve_stats", "accfem_solve_admm_iterations", "accfem_set_precision",
                 "accfem_batch_autotune", "accfem_batch_tuning", "accfem_set_element_modulus",
                 "accfem_set_frame_mode", "accfem_set_contact_solver", "accfem_batch_time_phase",
                 "accfem_set_contact_model"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t)


def accfem_default_options(**overrides):
    lib = load()
    o = accfem_options()
    lib.accfem_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def accfem_status_string(s):
    return load().accfem_status_string(int(s)).decode()


class AccFem:
    """One handle (robot + lumen resident on the current CUDA device)."""

    def __init__(self, robot, lumen, options=None, **overrides):
        lib = load()
        self._lib = lib
        self.robot = robot
        self.M = int(robot.n_elements)
        self.N = self.M + 1
        self._angles = np.ascontiguousarray(robot.cable_angles, dtype=np.float64)
        self._V = np.ascontiguousarray(np.asarray(lumen.vertices, dtype=np.float64).reshape(-1, 3))
        self._T = np.ascontiguousarray(np.asarray(lumen.triangles, dtype=np.int32).reshape(-1, 3))
        rd = accfem_robot_desc(robot.length, robot.outer_radius, robot.inner_radius, robot.youngs_modulus,
                               robot.poisson_ratio, self.M, len(self._angles), robot.cable_radius,
                               _ptr(self._angles))
        ld = accfem_lumen_desc(_ptr(self._V), len(self._V), _ptr(self._T, _ip), len(self._T),
                               (ctypes.c_double * 3)(*lumen.entrance_point), (ctypes.c_double * 3)(*lumen.entrance_dir),
                               (ctypes.c_double * 3)(*lumen.entrance_up))
        opt = options if options is not None else accfem_default_options(**overrides)
        self.options = opt
        h = ctypes.c_void_p()
        st = lib.accfem_create(ctypes.byref(rd), ctypes.byref(ld), ctypes.byref(opt), ctypes.byref(h))
        if st != OK:
            raise RuntimeError("accfem_create failed: %s" % accfem_status_string(st))
        self.h = h
        self.cap = int(opt.max_contacts)
        self._pos = np.zeros((self.N, 3))
        self._quat = np.zeros((self.N, 4))
        self._cn = np.zeros(self.cap, np.int32)
        self._ct = np.zeros(self.cap, np.int32)
        self._cp = np.zeros((self.cap, 3))
        self._cnrm = np.zeros((self.cap, 3))
        self._cf = np.zeros(self.cap)
        if getattr(robot, "element_youngs", None) is not None:
            st = self.accfem_set_element_modulus(robot.element_youngs)
            if st != OK:
                self.close()
                raise RuntimeError("accfem_set_element_modulus failed: %s" % accfem_status_string(st))

    def close(self):
        if getattr(self, "h", None):
            self._lib.accfem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _result_struct(self):
        return accfem_result(_ptr(self._pos), _ptr(self._quat), self.cap, 0, _ptr(self._cn, _ip), _ptr(self._ct, _ip),
                             _ptr(self._cp), _ptr(self._cnrm), _ptr(self._cf))

    def _pack(self, st, r):
        m = min(int(r.n_contacts), self.cap)
        return {"status": int(st), "node_pos": self._pos.copy(), "node_quat": self._quat.copy(),
                "n_contacts": int(r.n_contacts),
                "contacts": [{"node": int(self._cn[i]), "tri": int(self._ct[i]), "point": self._cp[i].copy(),
                              "normal": self._cnrm[i].copy(), "force": float(self._cf[i])} for i in range(m)],
                "base_reaction": np.array(r.base_reaction[:]), "newton_iters": int(r.newton_iters),
                "contact_iters": int(r.contact_iters), "residual": float(r.residual),
                "error": self._lib.accfem_last_error(self.h).decode()}

    @staticmethod
    def _warm(warm):
        if warm is None:
            return None, None
        pos = np.ascontiguousarray(warm[0], dtype=np.float64)
        quat = np.ascontiguousarray(warm[1], dtype=np.float64)
        return accfem_state(_ptr(pos), _ptr(quat)), (pos, quat)

    def accfem_solve(self, tensions, insertion, warm=None):
        t = np.ascontiguousarray(tensions, dtype=np.float64)
        ws, keep = self._warm(warm)
        r = self._result_struct()
        st = self._lib.accfem_solve(self.h, _ptr(t), float(insertion), ctypes.byref(ws) if ws else None, ctypes.byref(r))
        return self._pack(st, r)

    def accfem_solve_tip_load(self, f, m, follower, insertion, warm=None):
        f = np.ascontiguousarray(f, dtype=np.float64)
        m = np.ascontiguousarray(m, dtype=np.float64)
        ws, keep = self._warm(warm)
        r = self._result_struct()
        st = self._lib.accfem_solve_tip_load(self.h, _ptr(f), _ptr(m), int(bool(follower)), float(insertion),
                                             ctypes.byref(ws) if ws else None, ctypes.byref(r))
        return self._pack(st, r)

    def accfem_solve_resident(self, device_tensions_ptr, insertion):
        it = ctypes.c_int32(0)
        st = self._lib.accfem_solve_resident(self.h, ctypes.c_void_p(int(device_tensions_ptr)), float(insertion),
                                             ctypes.byref(it))
        return int(st), int(it.value)

    def accfem_get_state(self):
        pos = np.zeros((self.N, 3))
        quat = np.zeros((self.N, 4))
        st = self._lib.accfem_get_state(self.h, _ptr(pos), _ptr(quat))
        if st != OK:
            raise RuntimeError("accfem_get_state failed: %s" % accfem_status_string(st))
        return pos, quat

    def accfem_reset(self):
        return int(self._lib.accfem_reset(self.h))

    def accfem_set_stream(self, stream_ptr):
        return int(self._lib.accfem_set_stream(self.h, ctypes.c_void_p(int(stream_ptr)) if stream_ptr else None))

    def accfem_transfer_bytes(self):
        a, b = ctypes.c_int64(0), ctypes.c_int64(0)
        self._lib.accfem_transfer_bytes(self.h, ctypes.byref(a), ctypes.byref(b))
        return int(a.value), int(b.value)

    def accfem_time_kernel(self, kernel, reps=20):
        us = ctypes.c_double(0.0)
        st = self._lib.accfem_time_kernel(self.h, int(kernel), int(reps), ctypes.byref(us))
        if st != OK:
            raise RuntimeError("accfem_time_kernel failed: %s" % self.accfem_last_error())
        return float(us.value)

    def accfem_time_kernel_graph(self, kernel, reps=20):
        us = ctypes.c_double(0.0)
        st = self._lib.accfem_time_kernel_graph(self.h, int(kernel), int(reps), ctypes.byref(us))
        if st != OK:
            raise RuntimeError("accfem_time_kernel_graph failed: %s" % self.accfem_last_error())
        return float(us.value)

    def accfem_detect_contacts_noalloc(self, node_pos, n_nodes, row_capacity, row_node, row_tri, row_point,
                                       row_normal, row_gap, n_rows, stream=0):
        """Device pointers (ints) throughout; see include/accfem.h.  Returns the status code."""
        v = lambda x: ctypes.c_void_p(int(x)) if x else None
        return int(self._lib.accfem_detect_contacts_noalloc(self.h, v(node_pos), int(n_nodes), int(row_capacity),
                                                            v(row_node), v(row_tri), v(row_point), v(row_normal),
                                                            v(row_gap), v(n_rows), v(stream)))

    def accfem_kernel_launches(self):
        return int(self._lib.accfem_kernel_launches(self.h))

    def accfem_set_precision(self, mode):
        return int(self._lib.accfem_set_precision(self.h, int(mode)))

    def accfem_set_contact_solver(self, solver):
        """CONTACT_ACTIVE_SET (default) or CONTACT_ADMM (OSQP's ADMM guess, then the exact polish)."""
        return int(self._lib.accfem_set_contact_solver(self.h, int(solver)))

    def accfem_set_contact_model(self, model):
        """CONTACT_NODE (default) or CONTACT_SEGMENT (Eq. 3-7 at any point of an element)."""
        return int(self._lib.accfem_set_contact_model(self.h, int(model)))

    def accfem_set_frame_mode(self, iters_per_frame):
        """Frame mode: at most iters_per_frame Newton iterations per solve, OK at the cap (0: off)."""
        return int(self._lib.accfem_set_frame_mode(self.h, int(iters_per_frame)))

    def accfem_set_element_modulus(self, youngs_modulus, n_elements=None):
        """Per-element Young's moduli (None: the robot's own everywhere)."""
        if youngs_modulus is None:
            return int(self._lib.accfem_set_element_modulus(self.h, None, self.M if n_elements is None else int(n_elements)))
        E = np.ascontiguousarray(youngs_modulus, dtype=np.float64)
        n = len(E) if n_elements is None else int(n_elements)
        if n > len(E):                     # the C side would read n entries
            return E_INVALID_ARG
        return int(self._lib.accfem_set_element_modulus(self.h, _ptr(E), n))

    def accfem_solve_stats(self):
        """(constraint rows, working-set rows, active rows, FP64-tangent fallback) of the last solve."""
        a, b, c, f = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
        self._lib.accfem_solve_stats(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(f))
        return int(a.value), int(b.value), int(c.value), int(f.value)

    def accfem_solve_admm_iterations(self):
        """ADMM iterations of the last solve (contact solver CONTACT_ADMM)."""
        v = ctypes.c_int32(0)
        self._lib.accfem_solve_admm_iterations(self.h, ctypes.byref(v))
        return int(v.value)

    def accfem_device_bytes(self):
        v = ctypes.c_int64(0)
        self._lib.accfem_device_bytes(self.h, ctypes.byref(v))
        return int(v.value)

    def accfem_last_error(self):
        return self._lib.accfem_last_error(self.h).decode()


class AccFemBatch:
    """A batch over AccFem members (accfem_batch_* in include/accfem.h): solves of all members advance
    together, one kernel launch per Newton phase; members start and finish solves independently."""

    def __init__(self, members):
        lib = load()
        self._lib = lib
        self.members = list(members)
        n = len(self.members)
        arr = (ctypes.c_void_p * n)(*[m.h.value for m in self.members])
        b = ctypes.c_void_p()
        st = lib.accfem_batch_create(ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), n, ctypes.byref(b))
        if st != OK:
            raise RuntimeError("accfem_batch_create failed: %s" % accfem_status_string(st))
        self.b = b
        self.n = n

    def close(self):
        if getattr(self, "b", None):
            self._lib.accfem_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def accfem_batch_begin(self, member, tensions, insertion):
        t = np.ascontiguousarray(tensions, dtype=np.float64)
        return int(self._lib.accfem_batch_begin(self.b, int(member), _ptr(t), float(insertion)))

    def accfem_batch_advance(self, max_iters):
        left = ctypes.c_int32(0)
        st = self._lib.accfem_batch_advance(self.b, int(max_iters), ctypes.byref(left))
        return int(st), int(left.value)

    def accfem_batch_poll(self, member):
        done, st, it = ctypes.c_int32(0), ctypes.c_int(0), ctypes.c_int32(0)
        self._lib.accfem_batch_poll(self.b, int(member), ctypes.byref(done), ctypes.byref(st), ctypes.byref(it))
        return bool(done.value), int(st.value), int(it.value)

    def accfem_batch_results(self, members):
        """Results of the last finished solves of `members` as dicts (same keys as AccFem.accfem_solve)."""
        members = [int(i) for i in members]
        k = len(members)
        rs = (accfem_result * max(k, 1))()
        for j, i in enumerate(members):
            rs[j] = self.members[i]._result_struct()
        sts = (ctypes.c_int * max(k, 1))()
        ids = np.ascontiguousarray(members, dtype=np.int32)
        self._lib.accfem_batch_results(self.b, _ptr(ids, _ip), k, rs, sts)
        out = []
        for j, i in enumerate(members):
            d = self.members[i]._pack(sts[j], rs[j])
            d["error"] = self.accfem_batch_last_error()
            out.append(d)
        return out

    def accfem_batch_solve(self, tensions, insertions, mask=None, results=True):
        """One solve of every (masked) member; tensions is (n, k <= 8), insertions (n,).  Returns
        (first status, per-member statuses, per-member result dicts or None)."""
        t = np.zeros((self.n, MAX_CABLES))
        ta = np.asarray(tensions, dtype=np.float64).reshape(self.n, -1)
        t[:, :ta.shape[1]] = ta
        ins = np.ascontiguousarray(insertions, dtype=np.float64)
        mk = None if mask is None else np.ascontiguousarray(mask, dtype=np.int32)
        sts = (ctypes.c_int * self.n)()
        rs = None
        if results:
            rs = (accfem_result * self.n)()
            for i, m in enumerate(self.members):
                rs[i] = m._result_struct()
        st = self._lib.accfem_batch_solve(self.b, _ptr(t), _ptr(ins), _ptr(mk, _ip) if mk is not None else None, sts, rs)
        statuses = [int(sts[i]) for i in range(self.n)]
        out = None
        if results:
            sel = range(self.n) if mask is None else [i for i in range(self.n) if mask[i]]
            out = {i: self.members[i]._pack(statuses[i], rs[i]) for i in sel}
        return int(st), statuses, out

    def accfem_batch_serve(self, arrivals, members, tensions, insertions, chunk_iters=4, hbm_cap_bytes=0,
                           full_results=False):
        """Serves the requests (arrays of equal length, arrival-sorted) in real time; returns a dict of
        numpy arrays: status, newton_iters, t_begin, t_end, latency, tip (k, 7), n_contacts, and the
        call's status; with full_results, also "results": one dict per request (keys as
        AccFem.accfem_solve) holding the full answer of that request's solve."""
        k = len(arrivals)
        req = np.zeros(max(k, 1), dtype=REQUEST_DTYPE)
        if k:
            ta = np.asarray(tensions, dtype=np.float64).reshape(k, -1)
            req["arrival"][:k] = arrivals
            req["member"][:k] = members
            req["cable_tensions"][:k, :ta.shape[1]] = ta
            req["insertion"][:k] = insertions
        resp = np.zeros(max(k, 1), dtype=RESPONSE_DTYPE)
        rs, bufs = None, None
        if full_results and k:
            rs = (accfem_result * k)()
            bufs = []
            for j in range(k):
                m = self.members[int(req["member"][j])]
                cap = m.cap
                b = {"pos": np.zeros((m.N, 3)), "quat": np.zeros((m.N, 4)), "cn": np.zeros(cap, np.int32),
                     "ct": np.zeros(cap, np.int32), "cp": np.zeros((cap, 3)), "cnrm": np.zeros((cap, 3)),
                     "cf": np.zeros(cap), "cap": cap}
                rs[j] = accfem_result(_ptr(b["pos"]), _ptr(b["quat"]), cap, 0, _ptr(b["cn"], _ip), _ptr(b["ct"], _ip),
                                      _ptr(b["cp"]), _ptr(b["cnrm"]), _ptr(b["cf"]))
                bufs.append(b)
        st = self._lib.accfem_batch_serve(self.b, req.ctypes.data_as(ctypes.POINTER(accfem_request)), k,
                                          int(chunk_iters), int(hbm_cap_bytes),
                                          resp.ctypes.data_as(ctypes.POINTER(accfem_response)), rs)
        resp = resp[:k]
        out = {"call_status": int(st), "status": resp["status"].copy(), "newton_iters": resp["newton_iters"].copy(),
               "t_begin": resp["t_begin"].copy(), "t_end": resp["t_end"].copy(), "tip": resp["tip"].copy(),
               "n_contacts": resp["n_contacts"].copy()}
        out["latency"] = out["t_end"] - np.asarray(arrivals, dtype=np.float64)
        if full_results:
            full = []
            for j in range(k):
                b, r = bufs[j], rs[j]
                m = min(int(r.n_contacts), b["cap"])
                full.append({"status": int(resp["status"][j]), "node_pos": b["pos"], "node_quat": b["quat"],
                             "n_contacts": int(r.n_contacts),
                             "contacts": [{"node": int(b["cn"][i]), "tri": int(b["ct"][i]), "point": b["cp"][i].copy(),
                                           "normal": b["cnrm"][i].copy(), "force": float(b["cf"][i])} for i in range(m)],
                             "base_reaction": np.array(r.base_reaction[:]), "newton_iters": int(r.newton_iters),
                             "contact_iters": int(r.contact_iters), "residual": float(r.residual)})
            out["results"] = full
        return out

    def accfem_batch_time_phase(self, kernel, reps=5):
        """(status, mean microseconds per launch after an L2 flush, free nodes covered) of one phase kernel
        on the plan of the next iteration (KERNEL_ELEMENT, KERNEL_COLLIDE or KERNEL_ASSEMBLE)."""
        us, items = ctypes.c_double(0.0), ctypes.c_int64(0)
        st = self._lib.accfem_batch_time_phase(self.b, int(kernel), int(reps), ctypes.byref(us), ctypes.byref(items))
        return int(st), float(us.value), int(items.value)

    def accfem_batch_autotune(self, trials):
        return int(self._lib.accfem_batch_autotune(self.b, int(trials)))

    def accfem_batch_tuning(self):
        """(variant in use or -1 while tuning, ms per Newton iteration of each of the 12 variants: grid
        divisor 2^(v % 4), element blocks of 2 << (v / 4) warps)."""
        v = ctypes.c_int32(0)
        ms = np.zeros(12)
        self._lib.accfem_batch_tuning(self.b, ctypes.byref(v), _ptr(ms))
        return int(v.value), ms

    def accfem_batch_set_stream(self, stream_ptr):
        return int(self._lib.accfem_batch_set_stream(self.b, ctypes.c_void_p(int(stream_ptr)) if stream_ptr else None))

    def accfem_batch_transfer_bytes(self):
        a, b = ctypes.c_int64(0), ctypes.c_int64(0)
        self._lib.accfem_batch_transfer_bytes(self.b, ctypes.byref(a), ctypes.byref(b))
        return int(a.value), int(b.value)

    def accfem_batch_kernel_launches(self):
        return int(self._lib.accfem_batch_kernel_launches(self.b))

    def accfem_batch_last_error(self):
        return self._lib.accfem_batch_last_error(self.b).decode()
