"""Measured issue-rate peaks of the GPU (include/mcpeaks.h): single-precision
FMA, 32-bit integer multiply-add, 32x32->64 multiply, special-function unit
and shared-memory bandwidth. Used to put the walk kernel's throughput in
context; the walk does not call them."""
import ctypes as C
import os

from . import build as _b

KINDS = {"ffma": 0, "imad": 1, "mufu": 2, "smem_bytes": 3, "imul_wide": 4}


def measure(device=None, iters=4096, reps=5):
    """Return {kind: best ops/s over reps} (ops = thread-level operations,
    or bytes for shared memory)."""
    import torch
    lib = C.CDLL(_b.PEAKS_LIB) if os.path.exists(_b.PEAKS_LIB) else None
    if lib is None:
        raise RuntimeError("peaks library missing: build first")
    lib.mc_peak_run.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                C.POINTER(C.c_double), C.c_void_p]
    lib.mc_peak_run.restype = C.c_int
    dev = torch.device(device if device is not None else "cuda")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads = sms * 8, 256
    sink = torch.empty(blocks * threads, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream(dev)
    out = {}
    for name, kind in KINDS.items():
        it = iters if name != "smem_bytes" else iters // 2
        best = 0.0
        for r in range(reps + 1):
            ops = C.c_double()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            rc = lib.mc_peak_run(kind, blocks, threads, it, C.c_void_p(sink.data_ptr()), C.byref(ops),
                                 C.c_void_p(st.cuda_stream))
            b.record(st)
            if rc != 0:
                raise RuntimeError("mc_peak_run(%s) failed: %d" % (name, rc))
            b.synchronize()
            if r:
                best = max(best, ops.value / (a.elapsed_time(b) * 1e-3))
        out[name] = best
    out["sms"] = sms
    return out
