"""Resource peaks of the GPU the DSES kernels are bound by (microbenchmarks).

    python -m paper_2502_00115_b300.peaks      # prints one JSON line

Shared-memory atomic increments/s over a vote-sized histogram (random bins,
one bin per bank, a single bin), FP32 FMA/s, and random 4-byte and 16-byte
gathers/s from L2-resident tables (8 MB: a 128^3 FP32 grid; 32 MB: its
corner-block copy); libdses_peaks.so is built by paper_2502_00115_b300.build.
"""
import ctypes
import json
import os

LIB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libdses_peaks.so")


def run(device=0, nbins=45 * 45 * 23, table_bytes=8 << 20, table16_bytes=32 << 20):
    if not os.path.exists(LIB):
        raise RuntimeError(f"{LIB} is missing: build it with python -m paper_2502_00115_b300.build")
    lib = ctypes.CDLL(LIB)
    lib.dses_peaks_run.restype = ctypes.c_int
    lib.dses_peaks_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_size_t, ctypes.c_size_t,
                                   ctypes.POINTER(ctypes.c_double)]
    out = (ctypes.c_double * 6)()
    rc = lib.dses_peaks_run(device, nbins, table_bytes, table16_bytes, out)
    if rc != 0:
        raise RuntimeError(f"dses_peaks_run failed with CUDA error {rc}")
    return {"smem_atomic_random_per_s": out[0], "smem_atomic_bank_distinct_per_s": out[1],
            "smem_atomic_same_bin_per_s": out[2], "ffma_per_s": out[3], "l2_gather_4B_per_s": out[4],
            "l2_gather_16B_per_s": out[5], "histogram_words": nbins, "gather_table_bytes": table_bytes,
            "gather16_table_bytes": table16_bytes}


if __name__ == "__main__":
    print(json.dumps(run()))
