"""The on-chip bandwidths the benchmark's roofline uses as peaks where the
spins stay on chip (probes/peak_probes.cu, built here with nvcc on demand):

* L2 stream read: every SM reads a 64 MiB buffer that stays in L2, float4 by
  float4 through L2 (ld.cg), many times over; bytes read / time.
* Shared-memory gathers: one CTA per SM, each thread making random 8-byte
  loads from 128 KB of its CTA's shared memory, eight in flight; bytes
  loaded / time.

Each probe runs in a few launch shapes and reports its best.

HBM and the tensor pipes are measured by other means (MEASURED_PEAKS.json).
Run ``python bench.py --probe-peaks`` on the GPU."""
from __future__ import annotations

import ctypes as C
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "probes", "peak_probes.cu")
LIB = os.path.join(HERE, "probes", "libpeak_probes.so")


def _load():
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        nvcc = "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"
        subprocess.run([nvcc, "-gencode=arch=compute_103a,code=sm_103a", "-O3", "-shared", "-Xcompiler", "-fPIC",
                        "-cudart", "shared", "-o", LIB, SRC], check=True)
    lib = C.CDLL(LIB)
    lib.probe_l2_read.argtypes = [C.c_void_p, C.c_size_t, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p]
    lib.probe_smem_gather.argtypes = [C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p]
    return lib


def measure(device=0, repeats=5):
    """Best of `repeats` timings of each probe, in GB/s."""
    import torch
    lib = _load()
    dev = torch.device("cuda", device)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    stream = torch.cuda.Stream(dev)
    buf = torch.zeros(64 << 20, dtype=torch.uint8, device=dev)
    sink = torch.zeros(1, dtype=torch.float32, device=dev)

    def timed(fn):
        best = float("inf")
        for _ in range(repeats):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rc = fn()
            b.record(stream)
            b.synchronize()
            if rc:
                raise RuntimeError(f"probe launch failed: CUDA error {rc}")
            best = min(best, a.elapsed_time(b) * 1e-3)
        return best

    s = C.c_void_p(stream.cuda_stream)
    reps = 40
    lib.probe_l2_read(buf.data_ptr(), buf.numel(), 1, sink.data_ptr(), 4 * n_sm, 512, s)  # bring it into L2
    l2 = {}
    for per_sm, threads in ((2, 1024), (4, 512), (8, 256), (8, 512)):
        t = timed(lambda: lib.probe_l2_read(buf.data_ptr(), buf.numel(), reps, sink.data_ptr(), per_sm * n_sm,
                                            threads, s))
        l2[f"{per_sm}x{threads}"] = reps * buf.numel() / t / 1e9
    rounds, gathers = 4096, 8
    sm = {}
    for threads in (512, 768, 1024):
        t = timed(lambda: lib.probe_smem_gather(rounds, sink.data_ptr(), n_sm, threads, s))
        sm[str(threads)] = n_sm * threads * rounds * gathers * 8 / t / 1e9
    return {"l2_stream_read_GBps": max(l2.values()), "smem_random_8B_gather_GBps": max(sm.values()),
            "l2_by_shape": l2, "smem_by_threads": sm, "sms": n_sm}
