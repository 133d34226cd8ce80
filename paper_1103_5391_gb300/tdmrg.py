"""ctypes binding of libtdmrg (include/tdmrg.h): same names, argument marshalling only.

Vectors are torch.complex128 CUDA tensors (device pointers); every step of the
path runs in the library's kernels.  Loading fails loudly when libtdmrg.so is
missing: there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtdmrg.so")

TDMRG_OK, TDMRG_EINVAL, TDMRG_ENOMEM, TDMRG_ESECTOR, TDMRG_ECUDA, TDMRG_ETIMEOUT, TDMRG_ESTATE = 0, -1, -2, -3, -4, -5, -6
TDMRG_LEFT, TDMRG_RIGHT = 0, 1
TDMRG_FP64, TDMRG_OZAKI_BF16 = 0, 1

EXPORTED = [
    "tdmrg_default_opts", "tdmrg_create", "tdmrg_destroy", "tdmrg_set_stream", "tdmrg_set_precision",
    "tdmrg_last_error", "tdmrg_set_block", "tdmrg_set_op", "tdmrg_set_hamiltonian", "tdmrg_set_coefficients", "tdmrg_sector_size",
    "tdmrg_apply_h", "tdmrg_apply_op", "tdmrg_evolve", "tdmrg_evolve_info", "tdmrg_ground_state", "tdmrg_direct_sum", "tdmrg_evolve_segments", "tdmrg_evolve_segments_info", "tdmrg_tst_weights",
    "tdmrg_rho_size", "tdmrg_density_matrix", "tdmrg_set_real_basis", "tdmrg_rho_eig", "tdmrg_truncate", "tdmrg_renormalize_op", "tdmrg_wft_right", "tdmrg_wft_left", "tdmrg_density_matrix_side", "tdmrg_rho_size_side", "tdmrg_rho_eig_side", "tdmrg_density_eig", "tdmrg_truncate_side", "tdmrg_enlarge_size", "tdmrg_enlarge", "tdmrg_enlarge_bonds", "tdmrg_set_op_adjoint", "tdmrg_expect", "tdmrg_overlap_op", "tdmrg_correlation",
    "tdmrg_launch_count", "tdmrg_alloc_count", "tdmrg_hpsi_flops", "tdmrg_hpsi_tensor_flops", "tdmrg_fp64_peak", "tdmrg_apply_h_static",
    "tdmrg_set_schedule", "tdmrg_probe_wait", "tdmrg_hpsi_thin_flops", "tdmrg_set_thin_dim", "tdmrg_eig_stats", "tdmrg_set_tile_m", "tdmrg_hpsi_tuning", "tdmrg_set_orth_per_sm",
    "tdmrg_server_create", "tdmrg_server_submit", "tdmrg_server_poll", "tdmrg_server_cancel", "tdmrg_server_stats", "tdmrg_server_set_batching", "tdmrg_server_batch_stats",
    "tdmrg_server_destroy", "tdmrg_server_last_error",
]
TDMRG_JOB_QUEUED, TDMRG_JOB_RUNNING, TDMRG_JOB_DONE, TDMRG_JOB_CANCELLED, TDMRG_JOB_FAILED = 0, 1, 2, 3, 4


class tdmrg_job(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("q_gs", ctypes.c_int * 2), ("psi_gs_d", ctypes.c_void_p),
                ("q", ctypes.c_int * 2), ("phi0_d", ctypes.c_void_p), ("tau", ctypes.c_double), ("n_v", ctypes.c_int),
                ("nk", ctypes.c_int), ("steps", ctypes.c_int), ("nobs", ctypes.c_int),
                ("obs_opL", ctypes.c_int32 * 16), ("obs_opR", ctypes.c_int32 * 16)]


class tdmrg_opts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("prec", ctypes.c_int),
                ("ozaki_slices", ctypes.c_int), ("nk_max", ctypes.c_int), ("breakdown_tol", ctypes.c_double),
                ("hbm_budget", ctypes.c_size_t)]


class TdmrgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tdmrg error {code}: {msg}")
        self.code = code


_lib = None


def load(path=LIB_PATH):
    """Load libtdmrg.so (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with __graft_entry__.build() (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    PI32, PD, PI64 = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
    sig = {
        "tdmrg_default_opts": (None, [ctypes.POINTER(tdmrg_opts)]),
        "tdmrg_create": (I, [ctypes.POINTER(P), ctypes.POINTER(tdmrg_opts)]),
        "tdmrg_destroy": (I, [P]),
        "tdmrg_set_stream": (I, [P, P]),
        "tdmrg_set_precision": (I, [P, I, I]),
        "tdmrg_last_error": (ctypes.c_char_p, [P]),
        "tdmrg_set_block": (I, [P, I, I, PI32, PI32]),
        "tdmrg_set_op": (I, [P, I, I, I, I, PI32, P, I]),
        "tdmrg_set_hamiltonian": (I, [P, I, I, I, PI32, PI32, P]),
        "tdmrg_set_coefficients": (I, [P, P]),
        "tdmrg_sector_size": (I, [P, I, I, PI64]),
        "tdmrg_apply_h": (I, [P, I, I, P, P]),
        "tdmrg_apply_op": (I, [P, I, I, I, I, P, I, I, P]),
        "tdmrg_evolve": (I, [P, I, I, P, I, PD, I, ctypes.POINTER(P)]),
        "tdmrg_evolve_info": (I, [P, ctypes.POINTER(I), PD, PD, PD]),
        "tdmrg_ground_state": (I, [P, I, I, P, I, I, PD]),
        "tdmrg_direct_sum": (I, [P, I, P, PI32, PI32, PI64]),
        "tdmrg_evolve_segments": (I, [P, I, I, P, I, PI64, I, PD, I, P]),
        "tdmrg_evolve_segments_info": (I, [P, I, I, I, I, ctypes.POINTER(I), PD]),
        "tdmrg_tst_weights": (I, [I, PD, PD]),
        "tdmrg_rho_size": (I, [P, PI64, PI64]),
        "tdmrg_density_matrix": (I, [P, I, PI32, ctypes.POINTER(P), PD, P]),
        "tdmrg_rho_eig": (I, [P, P, P, P]),
        "tdmrg_set_real_basis": (I, [P, I]),
        "tdmrg_truncate": (I, [P, P, I, P, P]),
        "tdmrg_wft_right": (I, [P, I, I, P, P, PI32, P, PI32, P, P]),
        "tdmrg_wft_left": (I, [P, I, I, P, P, PI32, P, PI32, P, P]),
        "tdmrg_density_matrix_side": (I, [P, I, I, PI32, P, PD, P]),
        "tdmrg_rho_size_side": (I, [P, I, PI64, PI64]),
        "tdmrg_rho_eig_side": (I, [P, I, P, P, P]),
        "tdmrg_density_eig": (I, [P, I, I, PI32, P, PD, P, P, P]),
        "tdmrg_truncate_side": (I, [P, I, P, I, P, P]),
        "tdmrg_renormalize_op": (I, [P, I, I, P, PI32, P, ctypes.POINTER(I)]),
        "tdmrg_enlarge_size": (I, [I, I, PI32, PI32, I, ctypes.POINTER(I), PI32, PI32, PI32, ctypes.POINTER(ctypes.c_int64)]),
        "tdmrg_enlarge": (I, [P, I, I, PI32, PI32, P, P, ctypes.c_double, ctypes.c_double, P, P, P, P]),
        "tdmrg_enlarge_bonds": (I, [P, I, I, PI32, PI32, P, I, P, P, ctypes.c_double, P, P, P, P, P]),
        "tdmrg_set_op_adjoint": (I, [P, I, I, I]),
        "tdmrg_eig_stats": (I, [P, I, PI32, PI64]),
        "tdmrg_set_tile_m": (I, [P, I]),
        "tdmrg_set_orth_per_sm": (I, [P, I]),
        "tdmrg_hpsi_tuning": (I, [P, I, I, PI32]),
        "tdmrg_expect": (I, [P, I, I, I, I, P, P]),
        "tdmrg_overlap_op": (I, [P, I, I, I, I, P, I, I, P, P]),
        "tdmrg_correlation": (I, [P, I, PI32, I, PI32, I, I, P, I, I, P, P]),
        "tdmrg_launch_count": (I, [P, PI64]),
        "tdmrg_alloc_count": (I, [P, PI64, PI64]),
        "tdmrg_set_schedule": (I, [P, I]),
        "tdmrg_set_thin_dim": (I, [P, I]),
        "tdmrg_hpsi_thin_flops": (I, [P, I, I, PD]),
        "tdmrg_probe_wait": (I, [P, I64]),
        "tdmrg_hpsi_flops": (I, [P, I, I, PD]),
        "tdmrg_hpsi_tensor_flops": (I, [P, I, I, PD]),
        "tdmrg_fp64_peak": (I, [I, PD, PD]),
        "tdmrg_apply_h_static": (I, [P, I, I, P, P]),
        "tdmrg_server_create": (I, [ctypes.POINTER(P), I, ctypes.c_size_t, I]),
        "tdmrg_server_submit": (I, [P, ctypes.POINTER(tdmrg_job), PI64]),
        "tdmrg_server_poll": (I, [P, ctypes.c_int64, ctypes.POINTER(I), ctypes.POINTER(I), P, P]),
        "tdmrg_server_cancel": (I, [P, ctypes.c_int64]),
        "tdmrg_server_set_batching": (I, [P, I, I]),
        "tdmrg_server_batch_stats": (I, [P, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_int64)]),
        "tdmrg_server_stats": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                                   ctypes.POINTER(ctypes.c_size_t)]),
        "tdmrg_server_destroy": (I, [P]),
        "tdmrg_server_last_error": (ctypes.c_char_p, [P, ctypes.c_int64]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(ctx, rc):
    if rc != TDMRG_OK:
        msg = load().tdmrg_last_error(ctx)
        raise TdmrgError(rc, msg.decode() if msg else "")
    return rc


def _i32(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_cuda:
            raise ValueError("device vectors must be CUDA tensors")
        if not t.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(int(t))


# ----------------------------------------------------------------------------- calls
def tdmrg_default_opts():
    o = tdmrg_opts()
    load().tdmrg_default_opts(ctypes.byref(o))
    return o


def tdmrg_create(opts=None, **kw):
    o = opts or tdmrg_default_opts()
    for k, v in kw.items():
        setattr(o, k, v)
    h = ctypes.c_void_p()
    _check(None, load().tdmrg_create(ctypes.byref(h), ctypes.byref(o)))
    return h


def tdmrg_destroy(ctx):
    return _check(ctx, load().tdmrg_destroy(ctx))


def tdmrg_set_stream(ctx, stream):
    return _check(ctx, load().tdmrg_set_stream(ctx, ctypes.c_void_p(stream)))


def tdmrg_set_precision(ctx, prec, slices=4):
    return _check(ctx, load().tdmrg_set_precision(ctx, prec, slices))


def tdmrg_last_error(ctx):
    m = load().tdmrg_last_error(ctx)
    return m.decode() if m else ""


def tdmrg_set_block(ctx, side, qn, dims):
    q, qp = _i32(np.asarray(qn).reshape(-1))
    d, dp = _i32(dims)
    return _check(ctx, load().tdmrg_set_block(ctx, side, len(d), qp, dp))


def tdmrg_set_op(ctx, side, op_id, odd, blocks):
    """blocks: list of ((out_up, out_dn), (in_up, in_dn), 2-D complex array)."""
    qn = []
    parts = []
    for qo, qi, blk in blocks:
        qn.extend([qo[0], qo[1], qi[0], qi[1]])
        parts.append(np.ascontiguousarray(np.asarray(blk, dtype=np.complex128)).reshape(-1))
    q, qp = _i32(qn if qn else [0])
    data = np.concatenate(parts) if parts else np.zeros(1, np.complex128)
    return _check(ctx, load().tdmrg_set_op(ctx, side, op_id, int(odd), len(blocks), qp,
                                           data.ctypes.data_as(ctypes.c_void_p), 0))


def tdmrg_set_op_device(ctx, side, op_id, odd, blk_qn, data_d):
    """Operator from device data: blk_qn a list of (out_up, out_dn, in_up, in_dn), data_d the blocks
    row-major, concatenated in that order (e.g. the outputs of tdmrg_enlarge or tdmrg_renormalize_op)."""
    q, qp = _i32(np.asarray(blk_qn, dtype=np.int32).reshape(-1) if len(blk_qn) else [0])
    return _check(ctx, load().tdmrg_set_op(ctx, side, op_id, int(odd), len(blk_qn), qp, _ptr(data_d), 1))


def tdmrg_set_hamiltonian(ctx, opHL, opHR, conns):
    """conns: list of (opL, opR, complex coeff)."""
    n = len(conns)
    oL, pL = _i32([c[0] for c in conns] or [0])
    oR, pR = _i32([c[1] for c in conns] or [0])
    co = np.array([complex(c[2]) for c in conns] or [0j], dtype=np.complex128)
    return _check(ctx, load().tdmrg_set_hamiltonian(ctx, opHL, opHR, n, pL, pR, co.ctypes.data_as(ctypes.c_void_p)))


def tdmrg_set_coefficients(ctx, coeff_d):
    """Connection coefficients read at run time from the device array coeff_d (None: static)."""
    return _check(ctx, load().tdmrg_set_coefficients(ctx, _ptr(coeff_d) if coeff_d is not None else None))


def tdmrg_sector_size(ctx, Q):
    n = ctypes.c_int64()
    _check(ctx, load().tdmrg_sector_size(ctx, Q[0], Q[1], ctypes.byref(n)))
    return n.value


def tdmrg_apply_h(ctx, Q, psi, out):
    return _check(ctx, load().tdmrg_apply_h(ctx, Q[0], Q[1], _ptr(psi), _ptr(out)))


def tdmrg_apply_op(ctx, opL, opR, Q_in, psi, Q_out, out):
    return _check(ctx, load().tdmrg_apply_op(ctx, opL, opR, Q_in[0], Q_in[1], _ptr(psi), Q_out[0], Q_out[1], _ptr(out)))


def tdmrg_evolve(ctx, Q, phi, times, nk, targets):
    t = np.ascontiguousarray(np.asarray(times, dtype=np.float64))
    arr = (ctypes.c_void_p * len(targets))(*[_ptr(x) for x in targets])
    return _check(ctx, load().tdmrg_evolve(ctx, Q[0], Q[1], _ptr(phi), len(t),
                                           t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nk, arr))


def tdmrg_ground_state(ctx, Q, psi, nk=16, restarts=20):
    """psi (device, sector Q): start vector in, ground state out; returns the energy."""
    e = ctypes.c_double()
    _check(ctx, load().tdmrg_ground_state(ctx, Q[0], Q[1], _ptr(psi), nk, restarts, ctypes.byref(e)))
    return e.value


def tdmrg_direct_sum(ctx, srcs, Qs):
    """Loads the direct sum of the sources' superblocks into ctx; returns (Qsum, segment offsets)."""
    arr = (ctypes.c_void_p * len(srcs))(*[x.value if hasattr(x, "value") else x for x in srcs])
    q, qp = _i32(np.asarray(Qs).reshape(-1))
    qs = np.zeros(2, np.int32)
    off = np.zeros(len(srcs) + 1, np.int64)
    _check(ctx, load().tdmrg_direct_sum(ctx, len(srcs), arr, qp, qs.ctypes.data_as(_PI32),
                                        off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return (int(qs[0]), int(qs[1])), [int(x) for x in off]


def tdmrg_evolve_segments(ctx, Q, phi, seg_len, times, nk, targets):
    t = np.ascontiguousarray(np.asarray(times, dtype=np.float64))
    sl = np.ascontiguousarray(np.asarray(seg_len, dtype=np.int64))
    arr = (ctypes.c_void_p * len(targets))(*[_ptr(x) for x in targets])
    return _check(ctx, load().tdmrg_evolve_segments(ctx, Q[0], Q[1], _ptr(phi), len(sl),
                                                    sl.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(t),
                                                    t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nk, arr))


def tdmrg_evolve_segments_info(ctx, Q, nk, nseg):
    n = np.zeros(nseg, np.int32)
    e = np.zeros(nseg, np.float64)
    _check(ctx, load().tdmrg_evolve_segments_info(ctx, Q[0], Q[1], nk, nseg, n.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                                  e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return n, e


def tdmrg_evolve_info(ctx, nk_max=32):
    n = ctypes.c_int()
    err = ctypes.c_double()
    a = np.zeros(nk_max)
    b = np.zeros(nk_max)
    _check(ctx, load().tdmrg_evolve_info(ctx, ctypes.byref(n), ctypes.byref(err),
                                         a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return n.value, err.value, a[:n.value], b[:n.value]


def tdmrg_tst_weights(n_v):
    wgs = ctypes.c_double()
    w = np.zeros(max(n_v, 1))
    _check(None, load().tdmrg_tst_weights(n_v, ctypes.byref(wgs), w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return wgs.value, w[:n_v].tolist()


def tdmrg_rho_size(ctx, side=0):
    r, e = ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, load().tdmrg_rho_size_side(ctx, side, ctypes.byref(r), ctypes.byref(e)))
    return r.value, e.value


def tdmrg_density_matrix(ctx, states, weights, rho, side=0):
    """states: list of (Q, tensor); side 0: rho_L, side 1: rho_R."""
    q, qp = _i32([x for Q, _ in states for x in Q])
    arr = (ctypes.c_void_p * len(states))(*[_ptr(v) for _, v in states])
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    if side == 0:
        return _check(ctx, load().tdmrg_density_matrix(ctx, len(states), qp, arr,
                                                       w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(rho)))
    return _check(ctx, load().tdmrg_density_matrix_side(ctx, side, len(states), qp, arr,
                                                        w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(rho)))


def tdmrg_density_eig(ctx, states, weights, rho, evals, evecs, side=0):
    """tdmrg_density_matrix and tdmrg_rho_eig in one call (states: list of (Q, tensor))."""
    q, qp = _i32([x for Q, _ in states for x in Q])
    arr = (ctypes.c_void_p * len(states))(*[_ptr(v) for _, v in states])
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    return _check(ctx, load().tdmrg_density_eig(ctx, side, len(states), qp, arr,
                                                w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(rho),
                                                _ptr(evals), _ptr(evecs)))


def tdmrg_set_real_basis(ctx, on):
    return _check(ctx, load().tdmrg_set_real_basis(ctx, 1 if on else 0))


def tdmrg_rho_eig(ctx, rho, evals, evecs, side=0):
    if side == 0:
        return _check(ctx, load().tdmrg_rho_eig(ctx, _ptr(rho), _ptr(evals), _ptr(evecs)))
    return _check(ctx, load().tdmrg_rho_eig_side(ctx, side, _ptr(rho), _ptr(evals), _ptr(evecs)))


def tdmrg_truncate(ctx, evals, m, kept, discarded=None, side=0):
    """kept (device int32, one per sector of the side) <- kept counts of the m-state truncation; discarded
    (device float64, optional) <- the dropped weight."""
    if side == 0:
        return _check(ctx, load().tdmrg_truncate(ctx, _ptr(evals), int(m), _ptr(kept), _ptr(discarded)))
    return _check(ctx, load().tdmrg_truncate_side(ctx, side, _ptr(evals), int(m), _ptr(kept), _ptr(discarded)))


def tdmrg_renormalize_op(ctx, side, op_id, U, kept, out):
    """out (device complex128) <- U^dag O U per kept block; kept: host sequence of kept counts of that
    side's sectors.  Returns the number of blocks written."""
    k, kp = _i32(kept)
    nb = ctypes.c_int()
    _check(ctx, load().tdmrg_renormalize_op(ctx, side, op_id, _ptr(U), kp, _ptr(out), ctypes.byref(nb)))
    return nb.value


def tdmrg_wft_right(ctx_from, Q, psi, U, kept, V, kept_next, ctx_to, out):
    """Transport psi (ctx_from, sector Q) to ctx_to's superblock when the centre moves one site right."""
    k, kp = _i32(kept)
    kn, knp = _i32(kept_next)
    return _check(ctx_from, load().tdmrg_wft_right(ctx_from, Q[0], Q[1], _ptr(psi), _ptr(U), kp, _ptr(V), knp,
                                                   ctx_to, _ptr(out)))


def tdmrg_wft_left(ctx_from, Q, psi, U, kept, V, kept_next, ctx_to, out):
    """Transport psi (ctx_from, sector Q) to ctx_to's superblock when the centre moves one site left."""
    k, kp = _i32(kept)
    kn, knp = _i32(kept_next)
    return _check(ctx_from, load().tdmrg_wft_left(ctx_from, Q[0], Q[1], _ptr(psi), _ptr(U), kp, _ptr(V), knp,
                                                  ctx_to, _ptr(out)))


_PI32 = ctypes.POINTER(ctypes.c_int32)


class _Blocks(ctypes.Structure):
    _fields_ = [("nblk", ctypes.c_int), ("blk_qn", ctypes.c_void_p), ("data_d", ctypes.c_void_p)]


def _blocks(qns, data):
    """tdmrg_blocks of a list of (out n_up, out n_dn, in n_up, in n_dn) and the device data."""
    q = np.ascontiguousarray(np.asarray(qns, dtype=np.int32).reshape(-1))
    b = _Blocks(len(q) // 4, q.ctypes.data_as(ctypes.c_void_p) if len(q) else None, _ptr(data))
    return b, q


def tdmrg_enlarge_size(side, qn, dim):
    """(sector quantum numbers, dims, blocks of c^dag'_up / c^dag'_dn, entries of H', c^dag'_up, c^dag'_dn)
    of the block (qn, dim) enlarged by one site on `side`."""
    q, qp = _i32(np.asarray(qn).reshape(-1))
    d, dp = _i32(dim)
    cap = 4 * len(d) + 4
    n = ctypes.c_int()
    qo = np.zeros(2 * cap, np.int32)
    do = np.zeros(cap, np.int32)
    nb = np.zeros(2, np.int32)
    ent = np.zeros(3, np.int64)
    _check(None, load().tdmrg_enlarge_size(side, len(d), qp, dp, cap, ctypes.byref(n),
                                           qo.ctypes.data_as(_PI32), do.ctypes.data_as(_PI32), nb.ctypes.data_as(_PI32),
                                           ent.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    k = n.value
    return [tuple(x) for x in qo[:2 * k].reshape(k, 2)], list(do[:k]), list(nb), list(ent)


def tdmrg_enlarge(ctx, side, qn, dim, H, cdag, t, U, H_out, cdag_out, n_out=None):
    """H = (block quantum numbers, device data) of H_K; cdag = [(qns, data) for up, down] of K's edge
    c^dag; H_out, cdag_out[2] (and optionally n_out[2], the new site's densities, laid out like H_out)
    device outputs sized by tdmrg_enlarge_size.  Returns the block quantum numbers of c^dag'_up and
    c^dag'_dn."""
    q, qp = _i32(np.asarray(qn).reshape(-1))
    d, dp = _i32(dim)
    _, _, nb, _ = tdmrg_enlarge_size(side, qn, dim)
    hb, hq = _blocks(*H)
    cb = (_Blocks * 2)()
    keep = []
    for s in range(2):
        b, bq = _blocks(*cdag[s])
        cb[s] = b
        keep.append(bq)
    outs = (ctypes.c_void_p * 2)(_ptr(cdag_out[0]), _ptr(cdag_out[1]))
    qouts = [np.zeros(4 * max(int(nb[s]), 1), np.int32) for s in range(2)]
    qptr = (ctypes.c_void_p * 2)(*[x.ctypes.data_as(ctypes.c_void_p) for x in qouts])
    nptr = (ctypes.c_void_p * 2)(_ptr(n_out[0]), _ptr(n_out[1])) if n_out is not None else None
    _check(ctx, load().tdmrg_enlarge(ctx, side, len(d), qp, dp, ctypes.byref(hb), cb, float(t), float(U), _ptr(H_out),
                                     outs, qptr, nptr))
    return [[tuple(x) for x in qouts[s][:4 * int(nb[s])].reshape(-1, 4)] for s in range(2)]


def tdmrg_enlarge_bonds(ctx, side, qn, dim, H, edges, ts, U, H_out, cdag_out, n_out=None, carry_out=None):
    """As tdmrg_enlarge with the new site bonded to K's edge and to the second site from it: edges =
    [[(qns, data) up, (qns, data) dn] per bonded site of K], ts their hoppings; carry_out[2] (device, sized
    like cdag_out) receives K's edge as the enlarged block's second site from the edge.  Returns the block
    quantum numbers of c^dag'_up and c^dag'_dn (also those of the carried operators)."""
    q, qp = _i32(np.asarray(qn).reshape(-1))
    d, dp = _i32(dim)
    _, _, nb, _ = tdmrg_enlarge_size(side, qn, dim)
    hb, hq = _blocks(*H)
    cb = (_Blocks * (2 * len(edges)))()
    keep = []
    for e, ops in enumerate(edges):
        for s in range(2):
            b, bq = _blocks(*ops[s])
            cb[2 * e + s] = b
            keep.append(bq)
    tv = np.ascontiguousarray(ts, dtype=np.float64)
    outs = (ctypes.c_void_p * 2)(_ptr(cdag_out[0]), _ptr(cdag_out[1]))
    qouts = [np.zeros(4 * max(int(nb[s]), 1), np.int32) for s in range(2)]
    qptr = (ctypes.c_void_p * 2)(*[x.ctypes.data_as(ctypes.c_void_p) for x in qouts])
    nptr = (ctypes.c_void_p * 2)(_ptr(n_out[0]), _ptr(n_out[1])) if n_out is not None else None
    cptr = (ctypes.c_void_p * 2)(_ptr(carry_out[0]), _ptr(carry_out[1])) if carry_out is not None else None
    _check(ctx, load().tdmrg_enlarge_bonds(ctx, side, len(d), qp, dp, ctypes.byref(hb), len(edges), cb,
                                           tv.ctypes.data_as(ctypes.c_void_p), float(U), _ptr(H_out), outs, qptr,
                                           nptr, cptr))
    return [[tuple(x) for x in qouts[s][:4 * int(nb[s])].reshape(-1, 4)] for s in range(2)]


def tdmrg_set_op_adjoint(ctx, side, op_id, src_id):
    return _check(ctx, load().tdmrg_set_op_adjoint(ctx, side, op_id, src_id))


def tdmrg_expect(ctx, opL, opR, Q, psi, out):
    return _check(ctx, load().tdmrg_expect(ctx, opL, opR, Q[0], Q[1], _ptr(psi), _ptr(out)))


def tdmrg_correlation(ctx, opsL, opsR, Q1, phi1, Q2, phi2, out):
    """out (device complex128, len(opsL) * len(opsR)) <- <phi1| opsL[i] opsR[j] |phi2>."""
    a, ap = _i32(opsL)
    b, bp = _i32(opsR)
    return _check(ctx, load().tdmrg_correlation(ctx, len(a), ap, len(b), bp, Q1[0], Q1[1], _ptr(phi1), Q2[0], Q2[1],
                                                _ptr(phi2), _ptr(out)))


def tdmrg_overlap_op(ctx, opL, opR, Q1, phi1, Q2, phi2, out):
    """out[0] = <phi1| opL opR |phi2> (phi2 in sector Q2, phi1 in the sector Q1 the operators lead to)."""
    return _check(ctx, load().tdmrg_overlap_op(ctx, opL, opR, Q1[0], Q1[1], _ptr(phi1), Q2[0], Q2[1], _ptr(phi2),
                                               _ptr(out)))


def tdmrg_eig_stats(ctx, nsec, side=0):
    """(sweeps, SM cycles) per sector (nsec sectors) of the last Jacobi seed of rho_eig on that side."""
    sw = np.zeros(nsec, np.int32)
    cy = np.zeros(nsec, np.int64)
    _check(ctx, load().tdmrg_eig_stats(ctx, side, sw.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                       cy.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return sw, cy


def tdmrg_set_orth_per_sm(ctx, k):
    return _check(ctx, load().tdmrg_set_orth_per_sm(ctx, k))


def tdmrg_set_tile_m(ctx, m):
    return _check(ctx, load().tdmrg_set_tile_m(ctx, m))


def tdmrg_hpsi_tuning(ctx, Q):
    """(tile M, schedule) of stage 1 and of stage 2 of the H psi plan of sector Q."""
    o = np.zeros(4, np.int32)
    _check(ctx, load().tdmrg_hpsi_tuning(ctx, Q[0], Q[1], o.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    return [(int(o[0]), int(o[1])), (int(o[2]), int(o[3]))]


def tdmrg_probe_wait(ctx, spins):
    return _check(ctx, load().tdmrg_probe_wait(ctx, spins))


def tdmrg_set_schedule(ctx, mode):
    return _check(ctx, load().tdmrg_set_schedule(ctx, mode))


def tdmrg_set_thin_dim(ctx, dim):
    return _check(ctx, load().tdmrg_set_thin_dim(ctx, dim))


def tdmrg_hpsi_thin_flops(ctx, Q):
    f = ctypes.c_double()
    _check(ctx, load().tdmrg_hpsi_thin_flops(ctx, Q[0], Q[1], ctypes.byref(f)))
    return f.value


def tdmrg_launch_count(ctx):
    n = ctypes.c_int64()
    _check(ctx, load().tdmrg_launch_count(ctx, ctypes.byref(n)))
    return n.value


def tdmrg_alloc_count(ctx):
    """(number, total bytes) of device allocations the context has made."""
    n, b = ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, load().tdmrg_alloc_count(ctx, ctypes.byref(n), ctypes.byref(b)))
    return n.value, b.value


def tdmrg_hpsi_flops(ctx, Q):
    f = ctypes.c_double()
    _check(ctx, load().tdmrg_hpsi_flops(ctx, Q[0], Q[1], ctypes.byref(f)))
    return f.value


def tdmrg_hpsi_tensor_flops(ctx, Q):
    f = ctypes.c_double()
    _check(ctx, load().tdmrg_hpsi_tensor_flops(ctx, Q[0], Q[1], ctypes.byref(f)))
    return f.value


def tdmrg_fp64_peak(device=0):
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(None, load().tdmrg_fp64_peak(device, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def tdmrg_apply_h_static(ctx, Q, psi, out):
    """H psi with scratch from the library's static device array (no allocation during the call)."""
    return _check(ctx, load().tdmrg_apply_h_static(ctx, Q[0], Q[1], _ptr(psi), _ptr(out)))


# ----------------------------------------------------------------------------- serving
def _scheck(srv, rc, job=-1):
    if rc != TDMRG_OK:
        m = load().tdmrg_server_last_error(srv, job)
        raise TdmrgError(rc, m.decode() if m else "")
    return rc


def tdmrg_server_create(device=0, hbm_budget=0, max_active=8):
    h = ctypes.c_void_p()
    _check(None, load().tdmrg_server_create(ctypes.byref(h), device, hbm_budget, max_active))
    return h


def tdmrg_server_submit(srv, ctx, Q_gs, psi_gs, Q, phi0, tau, n_v, nk, steps, observables=()):
    """observables: list of (opL, opR) measured after every step."""
    j = tdmrg_job()
    j.ctx = ctx.value if hasattr(ctx, "value") else ctx
    j.q_gs[0], j.q_gs[1] = Q_gs
    j.psi_gs_d = psi_gs.data_ptr()
    j.q[0], j.q[1] = Q
    j.phi0_d = phi0.data_ptr()
    j.tau, j.n_v, j.nk, j.steps = tau, n_v, nk, steps
    j.nobs = len(observables)
    for k, (a, b) in enumerate(observables):
        j.obs_opL[k], j.obs_opR[k] = a, b
    jid = ctypes.c_int64()
    _scheck(srv, load().tdmrg_server_submit(srv, ctypes.byref(j), ctypes.byref(jid)))
    return jid.value


def tdmrg_server_poll(srv, job_id, steps=0, nobs=0):
    """(status, steps_done, observables [steps_done x nobs] complex, step_ms [steps_done])."""
    st, done = ctypes.c_int(), ctypes.c_int()
    obs = np.zeros(max(steps * nobs, 1), dtype=np.complex128)
    ms = np.zeros(max(steps, 1), dtype=np.float32)
    _scheck(srv, load().tdmrg_server_poll(srv, job_id, ctypes.byref(st), ctypes.byref(done),
                                          obs.ctypes.data_as(ctypes.c_void_p) if steps * nobs else None,
                                          ms.ctypes.data_as(ctypes.c_void_p) if steps else None))
    n = done.value
    return st.value, n, obs[: n * nobs].reshape(n, nobs) if nobs else None, ms[:n]


def tdmrg_server_cancel(srv, job_id):
    return _scheck(srv, load().tdmrg_server_cancel(srv, job_id))


def tdmrg_server_stats(srv):
    q, r, f, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
    _scheck(srv, load().tdmrg_server_stats(srv, ctypes.byref(q), ctypes.byref(r), ctypes.byref(f), ctypes.byref(b)))
    return q.value, r.value, f.value, b.value


def tdmrg_server_set_batching(srv, max_group, window_us=2000):
    return _scheck(srv, load().tdmrg_server_set_batching(srv, max_group, window_us))


def tdmrg_server_batch_stats(srv):
    g, n = ctypes.c_int(), ctypes.c_int64()
    _scheck(srv, load().tdmrg_server_batch_stats(srv, ctypes.byref(g), ctypes.byref(n)))
    return g.value, n.value


def tdmrg_server_destroy(srv):
    return load().tdmrg_server_destroy(srv)


def tdmrg_server_last_error(srv, job_id=-1):
    m = load().tdmrg_server_last_error(srv, job_id)
    return m.decode() if m else ""
