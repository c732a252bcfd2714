"""ctypes binding of libspectau.so (argument marshalling only).

Every entry point of ``include/spectau.h`` is exposed under the same name.
Loading fails loudly when the library has not been built: there is no
Python or CPU fallback for any part of the step.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspectau.so")

SP_OK, SP_ERR_ARG, SP_ERR_CUDA, SP_ERR_OOM = 0, -1, -2, -3
SP_ERR_SINGULAR, SP_ERR_NOT_FACTORED, SP_ERR_NONFINITE = -4, -5, -6
SP_ERR_TIMEOUT, SP_ERR_STATE = -7, -8
STATUS_NAMES = {0: "SP_OK", -1: "SP_ERR_ARG", -2: "SP_ERR_CUDA", -3: "SP_ERR_OOM",
                -4: "SP_ERR_SINGULAR", -5: "SP_ERR_NOT_FACTORED", -6: "SP_ERR_NONFINITE",
                -7: "SP_ERR_TIMEOUT", -8: "SP_ERR_STATE"}
SP_FOURIER, SP_CHEBYSHEV = 0, 1
SP_RK222, SP_SBDF1, SP_SBDF2, SP_RK111, SP_RK443, SP_SBDF3, SP_SBDF4, SP_CNAB1, SP_CNAB2 = range(9)
SCHEMES = {"RK222": SP_RK222, "SBDF1": SP_SBDF1, "SBDF2": SP_SBDF2, "RK111": SP_RK111, "RK443": SP_RK443,
           "SBDF3": SP_SBDF3, "SBDF4": SP_SBDF4, "CNAB1": SP_CNAB1, "CNAB2": SP_CNAB2}
# implicit solves per step
STAGES = {"RK222": 2, "SBDF1": 1, "SBDF2": 1, "RK111": 1, "RK443": 4, "SBDF3": 1, "SBDF4": 1}
SP_PREC_FP64, SP_PREC_MIXED = 0, 1
SP_OP_ID, SP_OP_DX, SP_OP_DY = 0, 1, 2
SP_SOLVE_AUTO, SP_SOLVE_WINDOW, SP_SOLVE_LANES, SP_SOLVE_SPIKE = 0, 1, 2, 3
SOLVE_KERNELS = {"auto": SP_SOLVE_AUTO, "window": SP_SOLVE_WINDOW, "lanes": SP_SOLVE_LANES, "spike": SP_SOLVE_SPIKE}

EXPORTS = (
    "sp_create", "sp_destroy", "sp_last_error", "sp_add_problem", "sp_set_layout",
    "sp_set_pencils", "sp_set_bilinear_rhs", "sp_factor", "sp_set_field", "sp_get_field",
    "sp_dz", "sp_step", "sp_step_graph", "sp_sync_status", "sp_transform", "sp_eval_rhs",
    "sp_get_band", "sp_set_timing", "sp_last_solve_time", "sp_transform_backward_static",
    "sp_step_batched", "sp_batch_tile", "sp_adjoint_init", "sp_step_adjoint", "sp_transform_adjoint",
    "sp_dz_adjoint", "sp_step_record", "sp_set_solve_kernel", "sp_get_solve_work",
    "sp_cfl_frequency", "sp_cfl_dt", "sp_eig_target", "sp_measure_fma_peak",
    "sp_set_spike_blocks", "sp_get_spike_blocks", "sp_set_z_transform", "sp_get_z_transform",
    "sp_solve_lbvp", "sp_eig_residual", "sp_batch_persistent",
    "sp_set_batch_persistent",
)


class sp_basis(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n_coeff", ctypes.c_int32),
                ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("dealias_num", ctypes.c_int32), ("dealias_den", ctypes.c_int32)]


class SpectauError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None

P = ctypes.c_void_p
I32P = ctypes.POINTER(ctypes.c_int32)
F64P = ctypes.POINTER(ctypes.c_double)
I = ctypes.c_int
I64 = ctypes.c_int64
D = ctypes.c_double

_SIGS = {
    "sp_create": [ctypes.POINTER(P), I, P],
    "sp_destroy": [P],
    "sp_add_problem": [P, I, ctypes.POINTER(sp_basis), I, I, I, ctypes.POINTER(I)],
    "sp_set_layout": [P, I, I32P, I32P, I32P, I32P, I32P, I32P, I, I32P, F64P],
    "sp_set_pencils": [P, I, I64, I64, I, I64, I32P, I32P, F64P, F64P],
    "sp_set_bilinear_rhs": [P, I, I, I32P, F64P, I32P, I32P, I32P, I32P],
    "sp_factor": [P, I, D],
    "sp_set_field": [P, I, I, P, I, ctypes.c_char],
    "sp_get_field": [P, I, I, P, I, ctypes.c_char],
    "sp_dz": [P, I, I, I],
    "sp_step": [P, I, D, I],
    "sp_step_graph": [P, I, D, I],
    "sp_sync_status": [P, ctypes.POINTER(I64)],
    "sp_transform": [P, I, P, P, I, I, I, I, I],
    "sp_eval_rhs": [P, I, P, ctypes.POINTER(I)],
    "sp_get_band": [P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)],
    "sp_get_solve_work": [P, I, ctypes.POINTER(D), ctypes.POINTER(D)],
    "sp_cfl_frequency": [P, I, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D)],
    "sp_cfl_dt": [D, D, D, D, D, D, D, D, ctypes.POINTER(D)],
    "sp_eig_target": [P, I, D, I, P, P, P],
    "sp_set_timing": [P, I, I],
    "sp_last_solve_time": [P, I, ctypes.POINTER(D), ctypes.POINTER(I)],
    "sp_transform_backward_static": [P, P, I, I, I, I, I, P, ctypes.c_char_p, I],
    "sp_step_batched": [P, I, ctypes.POINTER(I), F64P, I, I],
    "sp_batch_tile": [P, I, ctypes.POINTER(I), ctypes.POINTER(I)],
    "sp_adjoint_init": [P, I],
    "sp_step_adjoint": [P, I, D, P, I, P],
    "sp_step_record": [P, I, D, I, P],
    "sp_set_solve_kernel": [P, I, I],
    "sp_transform_adjoint": [P, I, P, P, I, I, I, I, I],
    "sp_dz_adjoint": [P, I, P, P],
    "sp_measure_fma_peak": [I, I, ctypes.POINTER(D)],
    "sp_set_spike_blocks": [P, I, I],
    "sp_get_spike_blocks": [P, I, ctypes.POINTER(I)],
    "sp_set_z_transform": [P, I, I],
    "sp_get_z_transform": [P, I, ctypes.POINTER(I)],
    "sp_solve_lbvp": [P, I, I, I32P, P],
    "sp_eig_residual": [P, I, ctypes.POINTER(D)],
    "sp_batch_persistent": [P, I, ctypes.POINTER(I), ctypes.POINTER(I)],
    "sp_set_batch_persistent": [P, I, ctypes.POINTER(I), I],
}
Z_TRANSFORMS = {"auto": 0, "fft": 1, "mma": 2}


def measure_fma_peak(device, precision):
    """Measured FMA throughput of the device in TFLOP/s (precision 'fp64' or 'fp32')."""
    out = D()
    st = lib().sp_measure_fma_peak(int(device), 0 if precision == "fp64" else 1, ctypes.byref(out))
    if st != SP_OK:
        raise SpectauError(st, "sp_measure_fma_peak failed")
    return out.value


def lib():
    """Load libspectau.so (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.sp_last_error.argtypes = [P]
        L.sp_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def check(ctx, status):
    if status != SP_OK:
        msg = lib().sp_last_error(ctx).decode() if ctx else ""
        raise SpectauError(status, msg)
    return status


def i32(a):
    return a.ctypes.data_as(I32P)


def f64(a):
    return a.ctypes.data_as(F64P)
