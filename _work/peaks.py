"""Measure the arithmetic peaks the roofline needs that the HBM/bf16 peak file lacks:
FP64, FP32, TF32 and BF16 GEMM throughput through torch (cuBLAS), best of 5.

  python -m paper_2607_05853_b300.peaks
"""
import json

import torch


def gemm_tflops(dtype, n, tf32=False, reps=5):
    torch.backends.cuda.matmul.allow_tf32 = tf32
    a = torch.randn(n, n, device="cuda", dtype=dtype)
    b = torch.randn(n, n, device="cuda", dtype=dtype)
    for _ in range(2):
        a @ b
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        a @ b
        e.record()
        torch.cuda.synchronize()
        best = min(best, s.elapsed_time(e))
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def main():
    out = {"fp64_gemm_tflops": gemm_tflops(torch.float64, 4096),
           "fp32_gemm_tflops": gemm_tflops(torch.float32, 8192),
           "tf32_gemm_tflops": gemm_tflops(torch.float32, 8192, tf32=True),
           "bf16_gemm_tflops": gemm_tflops(torch.bfloat16, 8192),
           "device": torch.cuda.get_device_name()}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
