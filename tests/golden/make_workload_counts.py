"""Writes workload_counts.json: algorithmic work per packet of the benchmark workloads,
counted by the CPU oracle (grid cells visited by all walks of a packet), used as the
per-unit figure of the roofline.  Calls only oracle/ and the scene generators.

    python tests/golden/make_workload_counts.py
"""
import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2406_15632_gb300 import scenes as S  # noqa: E402

N = 1 << 18


def peel_left_out(prob, log, eps):
    """Mean over all packets of the peel-off cells a walk may leave out at tolerance eps."""
    ok = log[:, 8] == 0
    th, ph = prob.theta_obs, prob.phi_obs
    k = [math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)]
    cells = O.ray_cells(prob, log[ok, :3], k, eps)
    return float((cells[:, 0] - cells[:, 1]).sum()) / len(log)


def main():
    out = {}
    prob = S.flared_disk_problem(n=256)
    _, log = O.trace_single(prob, 1, N, log=True)
    out["flared_disk_single_scattering"] = {
        "cells_per_packet": float(log[:, 9].mean()),
        # the walks a tracer must take when rays whose tau_1 lies below tau_min are known
        # not to scatter without walking them (they count as no cells)
        "cells_per_packet_scattering_rays": float((log[:, 9] * (log[:, 8] != 1)).mean()),
        # and when the march to the scattering point does not walk again the cells of the
        # first walk that lie before it (each cell of the ray is walked once, plus the peel-off)
        "cells_per_packet_scattering_rays_single_pass": float(((log[:, 9] - log[:, 10]) * (log[:, 8] != 1)).mean()),
        # and when each peel-off walk ends once the depth still ahead is at most 2^-24 (the
        # FP32 tolerance of the tracer's tail maps): the cells it must visit
        "cells_per_packet_scattering_rays_single_pass_tail": float(
            ((log[:, 9] - log[:, 10]) * (log[:, 8] != 1)).mean() - peel_left_out(prob, log, 2.0 ** -24)),
        "packets": N,
        "contributing_fraction": float((log[:, 8] == 0).mean()),
        "note": "256^3 flared disk, point source, Sobol indices 1..2^18, all three walks per packet",
    }
    clumpy = S.clumpy_problem(n=128)
    n_multi = 1 << 14
    cells = O.multiple_cells(clumpy, n_multi, n_multi)
    out["clumpy_multiple_scattering"] = {
        "cells_per_packet": float(cells[:, 0].mean()),
        # without the forced steps' second passes over cells of their first walks
        "cells_per_packet_single_pass": float((cells[:, 0] - cells[:, 1]).mean()),
        "packets": n_multi,
        "note": "128^3 clumpy envelope, 20 orders, forced, roulette 1e-4, Sobol indices 2^14..2^15-1, "
                "all walks of all orders per packet",
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workload_counts.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
