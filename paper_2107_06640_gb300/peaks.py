"""Measure this GPU's peak rates for the roofline denominators and write
them to profiles/peaks.md (a table and one JSON line that bench.py reads).

    python -m paper_2107_06640_gb300.peaks            # on a GPU

Probes (libadg.so, adg_measure_peak): a tcgen05 kind::tf32 MMA loop (dense
TF32 tensor rate; every 3xTF32 split product costs three of its MMAs), an
FP32 and an FP64 fused-multiply-add loop on the CUDA cores.  Each is timed
with CUDA events over `reps` launches of about 20 ms (a few seconds in all),
with nvidia-smi sampling the SM clock meanwhile.
"""

import json
import os
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
OUT = os.path.join(ROOT, "profiles", "peaks.md")
KINDS = {0: ("tf32_tensor_tflops", "tcgen05.mma kind::tf32, M=128 N=256 K=8, FP32 accumulation, 1 CTA/SM"),
         1: ("fp32_fma_tflops", "FP32 FFMA, 8 independent chains per thread, 8 x 256 threads per SM"),
         2: ("fp64_fma_tflops", "FP64 DFMA, 8 independent chains per thread, 8 x 256 threads per SM")}
REPS = {0: 100, 1: 100, 2: 60}


def measure(device=0):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    from paper_2107_06640_gb300 import _lib, build
    build.build()
    import torch
    res = {"device_name": torch.cuda.get_device_name(device),
           "sm_count": torch.cuda.get_device_properties(device).multi_processor_count}
    rows = []
    for kind, (key, what) in KINDS.items():
        with bench.ClockSampler(os.path.join(tempfile.gettempdir(), f"clocks_peak{kind}.csv")) as cs:
            flops, ms = _lib.adg_measure_peak(kind, device, REPS[kind])
        clk = cs.summary(device)
        res[key] = flops / (ms * 1e-3) / 1e12
        res[key + "_clock"] = clk
        rows.append((key, what, res[key], ms, clk))
    return res, rows


def write(res, rows, path=OUT):
    lines = ["# Measured peak rates (roofline denominators)", "",
             "Command: `python -m paper_2107_06640_gb300.peaks` (runs `adg_measure_peak` of libadg.so; "
             "CUDA events over the timed launches, nvidia-smi clock samples every 200 ms meanwhile).", "",
             f"GPU: {res['device_name']}, {res['sm_count']} SMs.", "",
             "| probe | what | TFLOP/s | timed ms | median SM MHz under load | throttle reasons |",
             "|---|---|---|---|---|---|"]
    for key, what, v, ms, clk in rows:
        lines.append(f"| `{key}` | {what} | {v:.1f} | {ms:.0f} | {clk.get('sm_mhz')} | "
                     f"{', '.join(clk.get('reasons', [])) or 'none'} |")
    lines += ["", "Used by `bench.py`: the 3xTF32 peak is `tf32_tensor_tflops / 3` (three TF32 MMAs per split "
              "product); the CUDA-core kernels' ALU peaks are `fp32_fma_tflops` and `fp64_fma_tflops`.", "",
              "```json", json.dumps({k: v for k, v in res.items() if not k.endswith("_clock")}), "```", ""]
    with open(path, "w") as f:
        f.write("\n".join(lines))


def load(path=OUT):
    """The JSON line of profiles/peaks.md, or None."""
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    if "```json" not in txt:
        return None
    return json.loads(txt.split("```json", 1)[1].split("```", 1)[0])


if __name__ == "__main__":
    r, rw = measure()
    write(r, rw)
    print(json.dumps({k: v for k, v in r.items() if not k.endswith("_clock")}))
