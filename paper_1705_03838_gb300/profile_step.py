"""Per-kernel device times of the time step on one of the seeded workloads.

    python paper_1705_03838_gb300/profile_step.py [workload] [precision] [steps]

workload: a key of inputs.WORKLOADS (default medium); precision: 0 FP64,
1 mixed (default 1); steps: timed steps (default 4).  Runs two untimed steps,
then `steps` steps with CUDA events around every kernel of the step graph
(timing option 1), and prints the average microseconds per launch of each
kernel and the wall time per step.  Small enough to run under a profiler.
"""
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

from paper_1705_03838_gb300 import build, inputs, opf  # noqa: E402


def main(argv):
    name = argv[1] if len(argv) > 1 else "medium"
    precision = int(argv[2]) if len(argv) > 2 else 1
    steps = int(argv[3]) if len(argv) > 3 else 4
    build.build()
    w = inputs.WORKLOADS[name]
    h = opf.opf_create(w["N"], w["K"], w["M"], w["m_p"], w["alpha"], w["Re"], w["dt"])
    opf.opf_set_option(h, "precision", precision)
    opf.opf_set_state(h, inputs.workload_state(name))
    opf.opf_step(h, 2)
    torch.cuda.synchronize()
    opf.opf_set_option(h, "timing", 1)
    opf.opf_kernel_times(h, reset=True)
    t = time.time()
    opf.opf_step(h, steps)
    torch.cuda.synchronize()
    wall = (time.time() - t) / steps
    kt = opf.opf_kernel_times(h, reset=True)
    for k, (ms, n) in kt.items():
        print(f"{k:10s} {ms * 1e3 / max(n, 1):8.2f} us per launch ({n} launches)")
    print(f"wall {wall * 1e3:.3f} ms per step (with per-kernel events)")
    print("energy", opf.opf_energy(h))
    opf.opf_destroy(h)


if __name__ == "__main__":
    main(sys.argv)
