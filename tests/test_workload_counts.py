"""The per-packet work figures of the roofline (tests/golden/workload_counts.json, written
by make_workload_counts.py from the oracle alone): each narrower count is a part of the
wider one, and the oracle's march count is a part of the cells its walks visit."""
import json
import os

import numpy as np

from oracle import oracle as O
from paper_2406_15632_gb300 import scenes as S

HERE = os.path.dirname(os.path.abspath(__file__))


def test_stored_counts_nest():
    c = json.load(open(os.path.join(HERE, "golden", "workload_counts.json")))
    d = c["flared_disk_single_scattering"]
    assert 0 < d["cells_per_packet_scattering_rays_single_pass_tail"] < d["cells_per_packet_scattering_rays_single_pass"]
    assert d["cells_per_packet_scattering_rays_single_pass"] < d["cells_per_packet_scattering_rays"]
    assert d["cells_per_packet_scattering_rays"] < d["cells_per_packet"]
    m = c["clumpy_multiple_scattering"]
    assert 0 < m["cells_per_packet_single_pass"] < m["cells_per_packet"]


def test_march_cells_are_a_prefix_of_the_first_walk():
    """Per packet of a small disk: the march to the scattering point visits at least one cell
    and no more than the other walks together (it retraces a prefix of the first walk's ray),
    and a packet that does not scatter marches nothing."""
    prob = S.flared_disk_problem(n=32, nx=16, ny=16)
    _, log = O.trace_single(prob, 1, 4096, log=True)
    marched, total, status = log[:, 10], log[:, 9], log[:, 8]
    assert np.all(marched[status == 1] == 0)
    s = status != 1
    assert np.all(marched[s] >= 1)
    assert np.all(marched[s] <= total[s] - marched[s])
