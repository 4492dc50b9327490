"""Split-TF32 factorizations for ncu captures of the tensor-core path.

  --case small  8192 x 8192 FP32 (256 MB, larger than L2), the mixed spectrum,
                b = 256, fixed rank 512 (two blocks): one launch each of the
                stream-K sketch and projection and of the update per block;
                for --set full captures of one kernel.
  --case mixed  the 32768 x 16384 split-TF32 workload (b = 256, eps =
                1e-3 ||A||_F): one warm-up factorization, then one inside
                cudaProfilerStart/Stop, for launch lists taken with
                ncu --profile-from-start off.
  --case fp32   the same for the 20000 x 16000 plain FP32 workload (b = 128,
                eps = 1e-2 ||A||_F)
  --case fp64   the same for the 2000 x 1000 FP64 workload (b = 50,
                eps = 1e-4 ||A||_F)
  --case bf16   the same for the BF16 storage leg (the mixed matrix stored
                in BF16, b = 256, eps = 1e-2 ||A||_F)
  --case small16  8192 x 8192 BF16 (128 MB), fixed rank 512 (two blocks), for
                --set full captures of the BF16 kernels
  --case batched  the same for the 512-matrix batch (b = 32, eps_t =
                1e-3 ||A_t||_F) through rqb_factor_batched
  --case batched64  the first 64 matrices of that batch (about 0.6 GB), for
                --set full captures of the grouped kernels
Usage: python -m paper_1503_07157_gb300.profile_case [--case small|mixed|fp32|fp64]
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", choices=["small", "small16", "mixed", "bf16", "fp32", "fp64", "batched", "batched64"], default="small")
    args = ap.parse_args()
    import torch
    import inputs
    from paper_1503_07157_gb300 import build, rqb
    build.build()
    if args.case == "small":
        m = n = 8192
        s = inputs.spectrum_mixed_config(min(m, n), knee=2000)
        A = inputs.usv_torch(m, n, s, 3, device="cuda", dtype=torch.float32)
        torch.cuda.synchronize()
        with rqb.Handle(torch.float32, prec=rqb.RQB_PREC_TF32X3, max_rank=512, fixed_rank=True) as h:
            _, _, k, rc = h.rqb_factor(A, 0.0, 256, 0, check=False)
            torch.cuda.synchronize()
    elif args.case == "small16":
        m = n = 8192
        s = inputs.spectrum_mixed_config(min(m, n), knee=2000)
        A32 = inputs.usv_torch(m, n, s, 3, device="cuda", dtype=torch.float32)
        A = torch.empty(n, m, dtype=torch.bfloat16, device="cuda").t()
        A.copy_(A32)
        del A32
        torch.cuda.synchronize()
        with rqb.Handle(torch.bfloat16, max_rank=512, fixed_rank=True) as h:
            _, _, k, rc = h.rqb_factor(A, 0.0, 256, 0, check=False)
            torch.cuda.synchronize()
    elif args.case in ("batched", "batched64"):
        mats, eps, _ = inputs.config_batched_torch(512 if args.case == "batched" else 64)
        torch.cuda.synchronize()
        with rqb.Handle(torch.float32) as h:
            h.rqb_factor_batched(mats, eps, 32, seed=0)
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
            out = h.rqb_factor_batched(mats, eps, 32, seed=0)
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
        k = sum(o[2] for o in out)
        rc = 0 if all(o[3] == rqb.RQB_OK for o in out) else 1
    else:
        import numpy as np
        if args.case in ("mixed", "bf16"):
            A, meta = inputs.config_mixed_torch()
            dt, prec, eps, b = torch.float32, rqb.RQB_PREC_TF32X3, meta["eps"], meta["b"]
            if args.case == "bf16":
                Ab = torch.empty(A.shape[1], A.shape[0], dtype=torch.bfloat16, device="cuda").t()
                Ab.copy_(A)
                del A
                torch.cuda.empty_cache()
                A, dt, prec, eps = Ab, torch.bfloat16, rqb.RQB_PREC_BF16, 10 * meta["eps"]
        elif args.case == "fp32":
            s = inputs.spectrum_poly(16000)
            A = inputs.usv_torch(20000, 16000, s, 2, device="cuda", dtype=torch.float32)
            dt, prec, eps, b = torch.float32, rqb.RQB_PREC_NATIVE, 1e-2 * float(np.sqrt(np.sum(s ** 2))), 128
        else:
            s = inputs.spectrum_fp64_config(1000)
            A = inputs.usv_torch(2000, 1000, s, 2, device="cuda", dtype=torch.float64)
            dt, prec, eps, b = torch.float64, rqb.RQB_PREC_NATIVE, 1e-4 * float(np.sqrt(np.sum(s ** 2))), 50
        torch.cuda.synchronize()
        with rqb.Handle(dt, prec=prec) as h:
            h.rqb_factor(A, eps, b, 0, check=False)
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
            _, _, k, rc = h.rqb_factor(A, eps, b, 0, check=False)
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
    print("case", args.case, "rc", rc, "k", k, flush=True)
    return 0 if rc == rqb.RQB_OK else 1


if __name__ == "__main__":
    sys.exit(main())
