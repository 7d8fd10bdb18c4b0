"""ctypes binding of the C ABI in ``include/lbm.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the scheme: all of that runs in the CUDA kernels of
``_build/liblbm.so``. Errors come back as ``LBMError`` carrying the status code
and ``lbm_last_error``. There is no CPU fallback: if the library cannot be
built or loaded, ``load()`` raises.

Arrays: numpy float64 arrays are host buffers; torch CUDA tensors are device
buffers (their ``data_ptr()`` is passed with on_device = 1). Field arrays are
[ny][nx], C-contiguous, float64.
"""
import ctypes
import os

from . import build as _build

LBM_OK = 0
LBM_ERR_INVALID = -1
LBM_ERR_UNSUPPORTED = -2
LBM_ERR_CUDA = -3
LBM_ERR_OOM = -4
LBM_ERR_NONFINITE = -5
LBM_ERR_TIMEOUT = -6

LBM_FP64, LBM_FP32, LBM_TC_BF16X3, LBM_TC_TF32X3, LBM_DF64, LBM_FP32_DWMOM = 0, 1, 2, 3, 4, 5
PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32, "tc_bf16x3": LBM_TC_BF16X3,
              "tc_tf32x3": LBM_TC_TF32X3, "df64": LBM_DF64, "fp32_dwmom": LBM_FP32_DWMOM}
BC = {"periodic": 0, "eq": 1, "reflect": 2, "extrap": 3, "wall": 4, "outflow": 5}
AUDIT_RING = 1024


class LBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("lbm status %d: %s" % (code, msg))
        self.code = code


class lbm_bc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("rho", ctypes.c_double), ("u", ctypes.c_double),
                ("v", ctypes.c_double), ("T", ctypes.c_double), ("split", ctypes.c_int),
                ("far_kind", ctypes.c_int), ("split0", ctypes.c_double),
                ("split_rate", ctypes.c_double)]


class lbm_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dt", ctypes.c_double),
                ("s", ctypes.c_double * 16), ("internal_dof", ctypes.c_int),
                ("precision", ctypes.c_int), ("bc", lbm_bc * 4),
                ("audit_every", ctypes.c_int)]


_LIB = None
_vp = ctypes.c_void_p
_ll = ctypes.c_longlong
_SIGS = {
    "lbm_create": (ctypes.c_int, [ctypes.POINTER(lbm_config), _vp, ctypes.POINTER(_vp)]),
    "lbm_set_init": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int]),
    "lbm_step": (ctypes.c_int, [_vp, _ll]),
    "lbm_moments": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int]),
    "lbm_destroy": (ctypes.c_int, [_vp]),
    "lbm_audit": (ctypes.c_int, [_vp, _vp]),
    "lbm_audit_log": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "lbm_status": (ctypes.c_int, [_vp, ctypes.POINTER(_ll), ctypes.POINTER(_ll)]),
    "lbm_step_count": (_ll, [_vp]),
    "lbm_get_populations": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(_ll), ctypes.c_int]),
    "lbm_set_populations": (ctypes.c_int, [_vp, _vp, _ll, ctypes.c_int]),
    "lbm_element_size": (ctypes.c_int, [_vp]),
    "lbm_last_error": (ctypes.c_char_p, [_vp]),
    "lbm_set_step_blocks": (ctypes.c_int, [_vp, ctypes.c_int]),
    "lbm_step_blocks": (ctypes.c_int, [_vp]),
    "lbm_autotune": (ctypes.c_int, [_vp, ctypes.c_int]),
}


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Loads liblbm.so (building it with nvcc first if it is missing or
    stale). Raises if it cannot be built or loaded."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("liblbm.so is not built (%s)" % _build.LIB)
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _err(ctx=None):
    return load().lbm_last_error(ctx).decode()


def _check(rc, ctx=None):
    if rc != LBM_OK:
        raise LBMError(rc, _err(ctx))
    return rc


def _ptr(a):
    """(pointer, on_device) of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), int(a.is_cuda)
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data, 0


def _dev(t):
    p, d = _ptr(t)
    if not d:
        raise ValueError("expected a CUDA tensor")
    return p


def make_config(nx, ny, dx, dy, dt, s, bc, precision="fp64", audit_every=0,
                internal_dof=0):
    """lbm_config from plain values; ``bc`` is four (kind, state) pairs for
    x-, x+, y-, y+ with kind a name in ``BC`` and state (rho, u, v, T) or
    None, or (kind, state, (far_kind, split0, split_rate)) for a split side:
    ``kind`` where the position along the side is <= split0 + split_rate t,
    ``far_kind`` beyond."""
    c = lbm_config()
    c.nx, c.ny = int(nx), int(ny)
    c.dx, c.dy, c.dt = float(dx), float(dy), float(dt)
    for k in range(16):
        c.s[k] = float(s[k])
    c.internal_dof = int(internal_dof)
    c.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    for k, side in enumerate(bc):
        kind, state = side[0], side[1]
        c.bc[k].kind = BC[kind] if isinstance(kind, str) else int(kind)
        if state is not None:
            c.bc[k].rho, c.bc[k].u, c.bc[k].v, c.bc[k].T = (float(x) for x in state)
        if len(side) > 2 and side[2] is not None:
            far, s0, s1 = side[2]
            c.bc[k].split = 1
            c.bc[k].far_kind = BC[far] if isinstance(far, str) else int(far)
            c.bc[k].split0, c.bc[k].split_rate = float(s0), float(s1)
    c.audit_every = int(audit_every)
    return c


def lbm_create(cfg, stream=None):
    """Returns the context handle (int). ``stream``: a cudaStream_t as int,
    a torch.cuda.Stream, or None."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    out = _vp()
    _check(load().lbm_create(ctypes.byref(cfg), _vp(stream or None), ctypes.byref(out)))
    return out.value


def lbm_set_init(ctx, rho, u, v, T):
    """f = f^eq(rho, u, v, T): four [ny][nx] fields, all host arrays
    (converted to C-contiguous float64) or all CUDA float64 tensors."""
    import numpy as np
    fields = [a if hasattr(a, "data_ptr") else np.ascontiguousarray(a, dtype=np.float64)
              for a in (rho, u, v, T)]
    ps = [_ptr(a) for a in fields]
    dev = {d for _, d in ps}
    if len(dev) != 1:
        raise ValueError("fields must all be host arrays or all device tensors")
    _check(load().lbm_set_init(ctx, *[p for p, _ in ps], dev.pop()), ctx)


def lbm_step(ctx, nsteps):
    _check(load().lbm_step(ctx, int(nsteps)), ctx)


def lbm_moments(ctx, rho=None, u=None, v=None, T=None):
    ps = [_ptr(a) for a in (rho, u, v, T)]
    dev = {d for p, d in ps if p is not None}
    if len(dev) > 1:
        raise ValueError("outputs must all be host arrays or all device tensors")
    _check(load().lbm_moments(ctx, *[p for p, _ in ps], dev.pop() if dev else 0), ctx)


def lbm_destroy(ctx):
    if ctx:
        _check(load().lbm_destroy(ctx))


def lbm_audit(ctx):
    buf = (ctypes.c_double * 4)()
    _check(load().lbm_audit(ctx, ctypes.cast(buf, _vp)), ctx)
    return list(buf)


def lbm_audit_log(ctx, max_entries=AUDIT_RING):
    tot = (ctypes.c_double * (4 * max_entries))()
    st = (ctypes.c_longlong * max_entries)()
    n = ctypes.c_int()
    _check(load().lbm_audit_log(ctx, ctypes.cast(tot, _vp), ctypes.cast(st, _vp),
                                int(max_entries), ctypes.byref(n)), ctx)
    k = n.value
    return [list(tot[4 * i:4 * i + 4]) for i in range(k)], list(st[:k])


def lbm_status(ctx):
    """(rc, first_bad_step, first_negT_step); rc is LBM_OK or
    LBM_ERR_NONFINITE (not raised), other codes raise."""
    a, b = _ll(), _ll()
    rc = load().lbm_status(ctx, ctypes.byref(a), ctypes.byref(b))
    if rc not in (LBM_OK, LBM_ERR_NONFINITE):
        _check(rc, ctx)
    return rc, a.value, b.value


def lbm_step_count(ctx):
    return int(load().lbm_step_count(ctx))


def lbm_get_populations(ctx, out):
    p, dev = _ptr(out)
    step = _ll()
    _check(load().lbm_get_populations(ctx, p, ctypes.byref(step), dev), ctx)
    return step.value


def lbm_set_populations(ctx, f, step):
    p, dev = _ptr(f)
    _check(load().lbm_set_populations(ctx, p, int(step), dev), ctx)


def lbm_element_size(ctx):
    return int(load().lbm_element_size(ctx))


def lbm_last_error(ctx=None):
    return _err(ctx)


def lbm_set_step_blocks(ctx, blocks):
    _check(load().lbm_set_step_blocks(ctx, int(blocks)), ctx)


def lbm_step_blocks(ctx):
    return int(load().lbm_step_blocks(ctx))


def lbm_autotune(ctx, launches=20):
    """Chooses the step's block count by timing; returns it."""
    _check(load().lbm_autotune(ctx, int(launches)), ctx)
    return lbm_step_blocks(ctx)


# ----------------------------------------------------------------------------
# Batches of quasi-1D tubes (include/lbm_batch.h)
# ----------------------------------------------------------------------------
class lbm_batch_config(ctypes.Structure):
    _fields_ = [("ntubes", ctypes.c_int), ("nx", ctypes.POINTER(ctypes.c_int)),
                ("dx", ctypes.POINTER(ctypes.c_double)), ("dt", ctypes.c_double),
                ("s", ctypes.POINTER(ctypes.c_double)), ("left", ctypes.POINTER(ctypes.c_double)),
                ("right", ctypes.POINTER(ctypes.c_double))]


_BATCH_SIGS = {
    "lbm_batch_create": (ctypes.c_int, [ctypes.POINTER(lbm_batch_config), _vp, ctypes.POINTER(_vp)]),
    "lbm_batch_set_init": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int]),
    "lbm_batch_step": (ctypes.c_int, [_vp, _ll]),
    "lbm_batch_moments": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int]),
    "lbm_batch_audit": (ctypes.c_int, [_vp, _vp]),
    "lbm_batch_status": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_set_tiling": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "lbm_batch_get_tiling": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_autotune": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_debug_skip_arrival": (ctypes.c_int, [_vp, ctypes.c_int, _ll]),
    "lbm_batch_step_count": (_ll, [_vp]),
    "lbm_batch_total_nodes": (ctypes.c_int, [_vp, ctypes.POINTER(_ll)]),
    "lbm_batch_destroy": (ctypes.c_int, [_vp]),
    "lbm_batch_last_error": (ctypes.c_char_p, [_vp]),
}
_SIGS.update(_BATCH_SIGS)
_SIGS.update({
    "lbm_audit_noalloc": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _ll,
                                         ctypes.c_double, ctypes.c_double, _vp, _vp]),
    "lbm_audit_noalloc_last_error": (ctypes.c_char_p, []),
    "lbm_set_fused_steps": (ctypes.c_int, [_vp, ctypes.c_int]),
    "lbm_fused_steps": (ctypes.c_int, [_vp]),
    "lbm_probe_fma_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_double,
                                          ctypes.POINTER(ctypes.c_double), _vp]),
})

PROBE_KINDS = {"fp64": 0, "fp32": 1, "fp32x2": 2}


def lbm_probe_fma_rate(kind, millis=50.0, stream=None):
    """Measured fused multiply-add rate of the current device (lane
    operations per second) for ``kind`` in PROBE_KINDS."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    out = ctypes.c_double()
    rc = load().lbm_probe_fma_rate(PROBE_KINDS[kind], float(millis), ctypes.byref(out),
                                   _vp(stream or None))
    if rc != LBM_OK:
        raise LBMError(rc, "lbm_probe_fma_rate failed")
    return out.value


def lbm_set_fused_steps(ctx, steps_per_launch):
    """Time steps per FP32 launch: 1 or 2 (temporal blocking)."""
    _check(load().lbm_set_fused_steps(ctx, int(steps_per_launch)), ctx)


def lbm_fused_steps(ctx):
    return int(load().lbm_fused_steps(ctx))
NOALLOC_MAX_BLOCKS = 4096


def lbm_audit_noalloc(f, precision, nx, ny, pitch, dx, dy, totals, stream=None):
    """Allocation-free conservation totals of a caller-owned device
    population tensor into a caller-owned device tensor of 4 doubles.

    The kernel trusts its pointers, so the tensors are checked here first:
    ``f`` a contiguous CUDA tensor on the current device whose dtype matches
    the precision (float64 for "fp64", float32 for "fp32") with at least
    16 * ny * pitch elements; ``totals`` a contiguous float64 CUDA tensor on
    the same device with at least 4 elements. A mismatch raises LBMError
    (LBM_ERR_INVALID) without touching the device."""
    import torch
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    want = {LBM_FP64: torch.float64, LBM_FP32: torch.float32}.get(prec)

    def bad(msg):
        raise LBMError(LBM_ERR_INVALID, "lbm_audit_noalloc: " + msg)

    for name, t in (("f", f), ("totals", totals)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
            bad("%s must be a contiguous CUDA tensor" % name)
        if t.device.index != torch.cuda.current_device():
            bad("%s is not on the current device" % name)
    if want is not None and f.dtype != want:
        bad("f has dtype %s, precision %s needs %s" % (f.dtype, precision, want))
    if int(nx) >= 1 and int(ny) >= 1 and f.numel() < 16 * int(ny) * int(pitch):
        bad("f holds %d elements, 16 x ny x pitch = %d needed" % (f.numel(), 16 * int(ny) * int(pitch)))
    if totals.dtype != torch.float64 or totals.numel() < 4:
        bad("totals must be float64 with at least 4 elements")
    rc = load().lbm_audit_noalloc(_dev(f), prec, int(nx), int(ny), int(pitch), float(dx),
                                  float(dy), _dev(totals), _vp(stream or None))
    if rc != LBM_OK:
        raise LBMError(rc, load().lbm_audit_noalloc_last_error().decode())
_KEEP = {}


def _bcheck(rc, b=None):
    if rc != LBM_OK:
        raise LBMError(rc, load().lbm_batch_last_error(b).decode())
    return rc


def lbm_batch_create(nx, dx, dt, s, left, right, stream=None):
    """nx: ints per tube; dx: spacing per tube; s: [ntubes][16]; left/right:
    [ntubes][4] (rho, u, v, T). Returns the batch handle."""
    import numpy as np
    nx = np.ascontiguousarray(nx, dtype=np.int32)
    dx = np.ascontiguousarray(dx, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    left = np.ascontiguousarray(left, dtype=np.float64)
    right = np.ascontiguousarray(right, dtype=np.float64)
    cfg = lbm_batch_config()
    cfg.ntubes = len(nx)
    cfg.nx = nx.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    cfg.dx = dx.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    cfg.dt = float(dt)
    cfg.s = s.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    cfg.left = left.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    cfg.right = right.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    out = _vp()
    _bcheck(load().lbm_batch_create(ctypes.byref(cfg), _vp(stream or None), ctypes.byref(out)))
    return out.value


def lbm_batch_set_init(b, rho, u, v, T):
    ps = [_ptr(a) for a in (rho, u, v, T)]
    dev = {d for _, d in ps}
    if len(dev) != 1:
        raise ValueError("fields must all be host arrays or all device tensors")
    _bcheck(load().lbm_batch_set_init(b, *[p for p, _ in ps], dev.pop()), b)


def lbm_batch_step(b, nsteps):
    _bcheck(load().lbm_batch_step(b, int(nsteps)), b)


def lbm_batch_moments(b, rho=None, u=None, v=None, T=None):
    ps = [_ptr(a) for a in (rho, u, v, T)]
    dev = {d for p, d in ps if p is not None}
    _bcheck(load().lbm_batch_moments(b, *[p for p, _ in ps], dev.pop() if dev else 0), b)


def lbm_batch_audit(b, ntubes):
    import numpy as np
    out = np.empty((ntubes, 4))
    _bcheck(load().lbm_batch_audit(b, out.ctypes.data), b)
    return out


def lbm_batch_status(b, ntubes):
    """(rc, first_bad[ntubes] (-1 = fine), nbad, timeout); LBM_ERR_TIMEOUT is
    returned in rc, not raised."""
    import numpy as np
    fb = np.empty(ntubes, dtype=np.int64)
    nbad, to = ctypes.c_int(), ctypes.c_int()
    rc = load().lbm_batch_status(b, fb.ctypes.data, ctypes.byref(nbad), ctypes.byref(to))
    if rc not in (LBM_OK, LBM_ERR_TIMEOUT):
        _bcheck(rc, b)
    return rc, fb, nbad.value, to.value


def lbm_batch_set_tiling(b, tile, threads):
    _bcheck(load().lbm_batch_set_tiling(b, int(tile), int(threads)), b)


def lbm_batch_get_tiling(b):
    t, th, bl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _bcheck(load().lbm_batch_get_tiling(b, ctypes.byref(t), ctypes.byref(th), ctypes.byref(bl)), b)
    return t.value, th.value, bl.value


def lbm_batch_autotune(b, trial_steps=20, cache_path=None):
    chosen = (ctypes.c_int * 2)()
    path = cache_path.encode() if cache_path else None
    _bcheck(load().lbm_batch_autotune(b, int(trial_steps), path, chosen), b)
    return chosen[0], chosen[1]


def lbm_batch_debug_skip_arrival(b, block, step):
    _bcheck(load().lbm_batch_debug_skip_arrival(b, int(block), int(step)), b)


def lbm_batch_step_count(b):
    return int(load().lbm_batch_step_count(b))


def lbm_batch_total_nodes(b):
    n = _ll()
    _bcheck(load().lbm_batch_total_nodes(b, ctypes.byref(n)), b)
    return n.value


def lbm_batch_destroy(b):
    if b:
        _bcheck(load().lbm_batch_destroy(b))


def lbm_batch_last_error(b=None):
    return load().lbm_batch_last_error(b).decode()


# ----------------------------------------------------------------------------
# Learned coarse-grid corrector (include/lbm_cnn.h)
# ----------------------------------------------------------------------------
CNN_NPARAMS = 30084
CNN_CHANNELS = (4, 32, 32, 32, 32, 4)

_SIGS.update({
    "lbm_cnn_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    "lbm_cnn_destroy": (ctypes.c_int, [_vp]),
    "lbm_cnn_set_params": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "lbm_cnn_get_params": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "lbm_cnn_set_adam": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "lbm_cnn_loss_grad": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(ctypes.c_double), _vp]),
    "lbm_cnn_train_step": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(ctypes.c_double)]),
    "lbm_cnn_correct": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]),
    "lbm_cnn_set_output_scale": (ctypes.c_int, [_vp, _vp]),
    "lbm_cnn_set_loss": (ctypes.c_int, [_vp, ctypes.c_int]),
    "lbm_cnn_residual_rms": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_restrict": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "lbm_cnn_last_error": (ctypes.c_char_p, [_vp]),
})


def _ccheck(rc, n=None):
    if rc != LBM_OK:
        raise LBMError(rc, load().lbm_cnn_last_error(n).decode())
    return rc


def lbm_cnn_create(H, W, stream=None):
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    out = _vp()
    _ccheck(load().lbm_cnn_create(int(H), int(W), _vp(stream or None), ctypes.byref(out)))
    return out.value


def lbm_cnn_destroy(n):
    if n:
        _ccheck(load().lbm_cnn_destroy(n))


def lbm_cnn_set_params(n, params):
    p, d = _ptr(params)
    _ccheck(load().lbm_cnn_set_params(n, p, d), n)


def lbm_cnn_get_params(n, out):
    p, d = _ptr(out)
    _ccheck(load().lbm_cnn_get_params(n, p, d), n)


def lbm_cnn_set_adam(n, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    _ccheck(load().lbm_cnn_set_adam(n, lr, beta1, beta2, eps), n)


def lbm_cnn_loss_grad(n, coarse, target, grads=None):
    """(loss, grads) for device field tensors [4][H][W]; grads: host float32
    array of CNN_NPARAMS (allocated when None)."""
    import numpy as np
    if grads is None:
        grads = np.empty(CNN_NPARAMS, dtype=np.float32)
    loss = ctypes.c_double()
    _ccheck(load().lbm_cnn_loss_grad(n, _dev(coarse), _dev(target), ctypes.byref(loss),
                                     grads.ctypes.data), n)
    return loss.value, grads


def lbm_cnn_train_step(n, coarse, target, want_loss=True):
    loss = ctypes.c_double()
    _ccheck(load().lbm_cnn_train_step(n, _dev(coarse), _dev(target),
                                      ctypes.byref(loss) if want_loss else None), n)
    return loss.value if want_loss else None


CNN_LOSS = {"mse": 0, "l1": 1}


def lbm_cnn_set_loss(n, kind):
    _ccheck(load().lbm_cnn_set_loss(n, CNN_LOSS[kind]), n)


def lbm_cnn_set_output_scale(n, scale):
    buf = (ctypes.c_double * 4)(*[float(x) for x in scale])
    _ccheck(load().lbm_cnn_set_output_scale(n, ctypes.cast(buf, _vp)), n)


def lbm_cnn_residual_rms(n, coarse, target):
    buf = (ctypes.c_double * 4)()
    _ccheck(load().lbm_cnn_residual_rms(n, _dev(coarse), _dev(target), ctypes.cast(buf, _vp)), n)
    return list(buf)


def lbm_cnn_correct(n, coarse, out, mass_tol=1e-2):
    fb = ctypes.c_int()
    _ccheck(load().lbm_cnn_correct(n, _dev(coarse), _dev(out), float(mass_tol), ctypes.byref(fb)), n)
    return bool(fb.value)


def lbm_restrict(fine, r, out, stream=None):
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    Hf, Wf = int(fine.shape[-2]), int(fine.shape[-1])
    _ccheck(load().lbm_restrict(_dev(fine), Hf, Wf, int(r), _dev(out), _vp(stream or None)))


# ----------------------------------------------------------------------------
# include/lbm_vn.h: linear (von Neumann) stability analysis of Sec. IV
# ----------------------------------------------------------------------------
class lbm_vn_case(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("u", ctypes.c_double), ("v", ctypes.c_double),
                ("T", ctypes.c_double), ("s", ctypes.c_double * 16)]


_SIGS.update({
    "lbm_vn_matrices": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, _vp, ctypes.c_int, _vp]),
    "lbm_vn_spectrum": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, _vp, _vp, ctypes.c_int,
                                       _vp, ctypes.POINTER(_ll)]),
    "lbm_eig16": (ctypes.c_int, [_vp, _ll, _vp, _vp, ctypes.c_int, _vp, ctypes.POINTER(_ll)]),
    "lbm_vn_last_error": (ctypes.c_char_p, []),
})


def _vn_check(rc):
    if rc != LBM_OK:
        raise LBMError(rc, load().lbm_vn_last_error().decode())


def _stream_ptr(stream):
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    return _vp(stream or None)


def vn_cases(states, rates):
    """float64 array [n][20] = (rho, u, v, T, s_1..s_16) per case, the memory
    layout of lbm_vn_case, from states [n][4] and rates [n][16]."""
    import numpy as np
    states = np.atleast_2d(np.asarray(states, dtype=np.float64))
    rates = np.atleast_2d(np.asarray(rates, dtype=np.float64))
    if states.shape[1] != 4 or rates.shape[1] != 16 or len(states) != len(rates):
        raise ValueError("states [n][4] and rates [n][16] expected")
    return np.ascontiguousarray(np.concatenate([states, rates], axis=1))


def _vn_args(cases, k):
    """(pointer, on_device, count) for the cases and the wave vectors; both
    host (numpy) or both device (torch CUDA)."""
    pc, dc = _ptr(cases)
    pk, dk = _ptr(k)
    if dc != dk:
        raise ValueError("cases and k must both be host or both be device arrays")
    if cases.shape[-1] != 20 or k.shape[-1] != 2:
        raise ValueError("cases [n][20] and k [nk][2] expected")
    return pc, pk, dc, int(cases.shape[0]), int(k.shape[0])


def lbm_vn_matrices(cases, k, dx, dy, dt, G=None, stream=None):
    """G of Sec. IV for every (case, wave vector). Host inputs: returns a
    complex128 array [ncases][nk][16][16]. Device inputs: G must be a float64
    CUDA tensor of [ncases * nk * 512] values (asynchronous)."""
    import numpy as np
    pc, pk, dev, nc, nk = _vn_args(cases, k)
    out = G if dev else np.empty((nc, nk, 16, 16), dtype=np.complex128)
    _vn_check(load().lbm_vn_matrices(_vp(pc), nc, _vp(pk), nk, float(dx), float(dy), float(dt),
                                     _vp(_ptr(out)[0]), dev, _stream_ptr(stream)))
    return out


def lbm_vn_spectrum(cases, k, dx, dy, dt, radius=None, omega=None, stream=None,
                    want_omega=True, count_nonconverged=True):
    """Eigenvalues omega of G and radius = max |omega| for every (case, wave
    vector). Host inputs: returns (radius [ncases][nk], omega [ncases][nk][16]
    complex or None, nonconverged). Device inputs: writes the given CUDA
    tensors (radius: ncases * nk doubles, omega: ncases * nk * 32 doubles)."""
    import numpy as np
    pc, pk, dev, nc, nk = _vn_args(cases, k)
    if not dev:
        radius = np.empty((nc, nk))
        omega = np.empty((nc, nk, 16), dtype=np.complex128) if want_omega else None
    nf = _ll(0)
    _vn_check(load().lbm_vn_spectrum(_vp(pc), nc, _vp(pk), nk, float(dx), float(dy), float(dt),
                                     _vp(_ptr(radius)[0]), _vp(_ptr(omega)[0]), dev,
                                     _stream_ptr(stream),
                                     ctypes.byref(nf) if count_nonconverged else None))
    return radius, omega, (nf.value if count_nonconverged else None)


def lbm_eig16(A, stream=None):
    """Eigenvalues of complex 16 x 16 matrices A [n][16][16] (host complex128):
    returns (omega [n][16] complex, radius [n], nonconverged)."""
    import numpy as np
    A = np.ascontiguousarray(A, dtype=np.complex128)
    if A.ndim != 3 or A.shape[1:] != (16, 16):
        raise ValueError("A [n][16][16] expected")
    n = A.shape[0]
    omega = np.empty((n, 16), dtype=np.complex128)
    radius = np.empty(n)
    nf = _ll(0)
    _vn_check(load().lbm_eig16(_vp(A.ctypes.data), n, _vp(omega.ctypes.data),
                               _vp(radius.ctypes.data), 0, _stream_ptr(stream), ctypes.byref(nf)))
    return omega, radius, nf.value
