"""Batched persistent launch: every instance of a batch equals the same instance traced
alone (bit for bit in fixed point, whatever the work decomposition), the FP64 batch
matches the oracle, and a captured CUDA graph replays to the same images."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2406_15632_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_2406_15632_gb300 import build as B
    from paper_2406_15632_gb300 import qmcrt

    B.build()
    qmcrt.load()
    return qmcrt


def small_batch(seed=3, n=12, source="sphere"):
    rng = np.random.default_rng(seed)
    out = []
    for j in range(n):
        c = int(2 ** rng.integers(9, 14))
        out.append(S.Instance(theta_obs=float(rng.uniform(0, math.pi)), albedo=float(rng.uniform(0.4, 0.9)),
                              g=float(rng.uniform(-0.3, 0.7)), kscale=float(rng.uniform(0.5, 4.0)), n_packets=c,
                              first_index=c if j % 3 else 1 + j))
    out.append(S.Instance(theta_obs=0.3, albedo=0.5, g=0.1, kscale=1.0, n_packets=0, first_index=1))
    return out


def base_problem(source="sphere", generator="sobol"):
    p = S.flared_disk_problem(n=32, nx=48, ny=40, generator=generator)
    if source == "sphere":
        p = p.replace(source="sphere", star_r=0.05, limb_u=0.6, emit_order="inverse")
    return p


def alone(Q, prob, I, fb, precision):
    import torch

    p = prob.replace(theta_obs=I.theta_obs, albedo=I.albedo, g=I.g, kscale=prob.kscale * I.kscale)
    sc = Q.Scene(p)  # with the tail map of its direction, as the batch's instance
    buf = sc.accum_buffer("i64")
    if I.n_packets:
        sc.trace(I.first_index, I.n_packets, buf, frac_bits=fb, precision=precision)
    torch.cuda.synchronize()
    return buf[0, 0].cpu().numpy()


@pytest.mark.parametrize("generator", ["sobol", "sobol_owen", "halton", "philox", "niederreiter", "faure"])
@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_batch_instances_equal_alone_runs(Q, generator, precision):
    import torch

    prob = base_problem(generator=generator)
    inst = small_batch()
    fb = 40
    B = Q.Batch(prob, inst, precision=precision, chunk_log2=10, frac_bits=fb, packets_per_thread=2)
    B.run()
    torch.cuda.synchronize()
    acc = B.accum.cpu().numpy()
    for k, I in enumerate(inst):
        assert np.array_equal(acc[k], alone(Q, prob, I, fb, precision)), k


@pytest.mark.parametrize("config", [(7, 64, 1, 1), (12, 128, 0, 8), (16, 256, 2, 4)])
def test_batch_result_does_not_depend_on_the_work_decomposition(Q, config):
    import torch

    prob = base_problem(source="point")
    inst = small_batch(seed=5)
    B = Q.Batch(prob, inst, chunk_log2=10, frac_bits=40)
    B.run()
    torch.cuda.synchronize()
    ref = B.accum.clone()
    B.set_config(*config)
    B.run()
    torch.cuda.synchronize()
    assert torch.equal(B.accum, ref)


def test_batch_fp64_matches_oracle(Q):
    import torch

    prob = base_problem()
    inst = small_batch(seed=7, n=5)
    B = Q.Batch(prob, inst, precision="f64", chunk_log2=9, frac_bits=48)
    B.run()
    torch.cuda.synchronize()
    out = B.out.cpu().numpy()
    for k, I in enumerate(inst):
        if not I.n_packets:
            assert np.all(out[k] == 0)
            continue
        p = prob.replace(theta_obs=I.theta_obs, albedo=I.albedo, g=I.g, kscale=I.kscale)
        ref = O.trace_single(p, I.first_index, I.n_packets) / I.n_packets
        assert np.linalg.norm(out[k] - ref) <= 1e-10 * np.linalg.norm(ref)


def test_batch_graph_replay_reproduces_the_run(Q):
    import torch

    prob = base_problem()
    inst = small_batch(seed=9)
    B = Q.Batch(prob, inst, chunk_log2=11, frac_bits=40)
    B.run()
    torch.cuda.synchronize()
    ref = B.out.clone()
    B.capture()
    for _ in range(2):
        B.out.zero_()
        B.replay()
        torch.cuda.synchronize()
        assert torch.equal(B.out, ref)


def test_sequential_path_gives_the_batch_images(Q):
    import torch

    prob = base_problem()
    inst = small_batch(seed=11)
    B = Q.Batch(prob, inst, chunk_log2=10, frac_bits=40)
    B.run()
    torch.cuda.synchronize()
    ref = B.accum.clone()
    B.run_each()
    torch.cuda.synchronize()
    assert torch.equal(B.accum, ref)
