"""Arithmetic peaks of the GPU that the HBM/BF16 peak file does not give.

The FP64 filter and the FP64 products are bound by the FP64 pipe, so their
roofline needs the FP64 rate; this times library GEMMs (torch.matmul, i.e.
cuBLAS) with CUDA events, best of five after two warm-ups, and prints one
JSON line.  Run on the GPU machine: ``python -m paper_1404_4161_gb300.peaks``.
"""
import json

import torch


def matmul_tflops(dtype, n, reps=5, complex_flops=False):
    a = torch.randn(n, n, device="cuda", dtype=dtype)
    b = torch.randn(n, n, device="cuda", dtype=dtype)
    for _ in range(2):
        a @ b
    torch.cuda.synchronize()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(reps):
        s.record()
        a @ b
        e.record()
        torch.cuda.synchronize()
        best = min(best, s.elapsed_time(e) / 1e3)
    return (8 if complex_flops else 2) * n ** 3 / best / 1e12


def main():
    p = torch.cuda.get_device_properties(0)
    out = {"device": torch.cuda.get_device_name(0), "sms": p.multi_processor_count,
           "torch": torch.__version__}
    out["float64_8192"] = matmul_tflops(torch.float64, 8192)
    out["complex128_4096"] = matmul_tflops(torch.complex128, 4096, complex_flops=True)
    torch.backends.cuda.matmul.allow_tf32 = False
    out["float32_8192"] = matmul_tflops(torch.float32, 8192)
    torch.backends.cuda.matmul.allow_tf32 = True
    out["tf32_8192"] = matmul_tflops(torch.float32, 8192)
    out["float16_8192"] = matmul_tflops(torch.float16, 8192)
    out["bfloat16_8192"] = matmul_tflops(torch.bfloat16, 8192)
    print(json.dumps({k: (round(v, 2) if isinstance(v, float) else v) for k, v in out.items()}))


if __name__ == "__main__":
    main()
