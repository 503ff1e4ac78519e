"""Time-sharded solves through the C ABI (destripe_plan_sharded /
destripe_solve_sharded) against the single-domain float64 oracle.

Two ranks run as two processes on the one GPU of the box, exchanging over gloo
through host memory (the library's all-reduce hook; the NCCL variant enqueues the
same exchange on the device).  No kernel of one rank waits on the other: every
exchange is a host-side collective between kernel launches.  Each rank holds a
contiguous slice of baselines and their samples; the gathered baselines and every
rank's global map must equal the oracle's at the parity bars (relative RMS 1e-5,
max |delta a| 1e-4 sigma), and a one-rank sharded solve must equal destripe_solve.
"""
import os
import socket

import numpy as np
import pytest
import torch

import oracle
import paper_1309_5609_gb300 as ds
from synth import make_problem

pytestmark = pytest.mark.gpu

CASES = {
    "qu": dict(n_t=120_000, nside=16, kinds=("q", "u"), baseline_len=97, flag_frac=0.0),
    "Iqu_flags": dict(n_t=90_001, nside=16, kinds=("I", "q", "u"), baseline_len=50,
                      flag_frac=0.05),
}


def _problem(case, precision):
    ydt = torch.float32 if precision == "mixed" else torch.float64
    return make_problem(seed=41, flag_mean_len=200, sky_sigma={"I": 10.0, "Q": 1.0, "U": 1.0},
                        y_dtype=ydt, keep_f64_trig=False, **CASES[case])


def _slice(prob, rank, world):
    L, n_b = prob.baseline_len, prob.n_b
    b_lo, b_hi = rank * n_b // world, (rank + 1) * n_b // world
    t_lo, t_hi = b_lo * L, min(b_hi * L, prob.n_t)
    return b_lo, b_hi, t_lo, t_hi


def _solve_rank(prob, rank, world, precision, allreduce):
    dev = torch.device("cuda:0")
    b_lo, b_hi, t_lo, t_hi = _slice(prob, rank, world)
    sl = slice(t_lo, t_hi)
    pix = prob.pix[sl].contiguous().to(dev)
    c = prob.c32[sl].contiguous().to(dev)
    s = prob.s32[sl].contiguous().to(dev)
    valid = None if prob.valid is None else prob.valid[sl].contiguous().to(dev)
    y = prob.y[:, sl].contiguous().to(dev)
    plan = ds.destripe_plan_sharded(pix, c, s, valid, nside=prob.nside, kinds=prob.kinds,
                                    baseline_len=prob.baseline_len, precision=precision,
                                    allreduce=allreduce)
    a = torch.zeros(plan.n_u, dtype=torch.float64, device=dev)
    st, it, rel = ds.destripe_solve_sharded(plan, y, a, tol=1e-10)
    m = torch.zeros(plan.n_c * plan.npix, dtype=torch.float64, device=dev)
    ds.destripe_map(plan, y, a, m)
    torch.cuda.synchronize()
    out = (st, it, rel, a.view(plan.n_o, -1).cpu().numpy(), m.cpu().numpy())
    plan.close()
    return out


def _rank_main(rank, world, port, case, precision, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        prob = _problem(case, precision)
        q.put((rank, _solve_rank(prob, rank, world, precision, ds.torch_allreduce())))
    except Exception as e:  # reported to the parent, never left hanging
        q.put((rank, repr(e)))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _oracle(prob):
    d = prob.numpy()
    op = oracle.make_plan(d["pix"], d["c"], d["s"], d["valid"], prob.nside, prob.kinds,
                          prob.baseline_len)
    return op, oracle.destripe(op, d["y"], tol=1e-10)


def rel_rms(a, b):
    a, b = np.asarray(a, float).ravel(), np.asarray(b, float).ravel()
    den = np.sqrt(np.mean(b ** 2))
    return float(np.sqrt(np.mean((a - b) ** 2)) / (den if den > 0 else 1.0))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", list(CASES))
def test_two_ranks_on_one_gpu_match_the_oracle(case, precision):
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, case, precision, q))
             for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        rank, out = q.get(timeout=600)
        res[rank] = out
    for p in procs:
        p.join(timeout=120)
    for r in range(2):
        assert not isinstance(res[r], str), res[r]
    prob = _problem(case, precision)
    op, ref = _oracle(prob)
    a = np.concatenate([res[0][3], res[1][3]], axis=1)
    for r in range(2):
        st, it, rel = res[r][:3]
        assert st == ds.DS_OK and rel < 1e-9, (r, st, it, rel)
    assert res[0][1] == res[1][1]  # both ranks ran the same iterations
    assert rel_rms(a.ravel(), ref["a"]) < 1e-5
    assert np.abs(a.ravel() - ref["a"]).max() < 1e-4
    for r in range(2):  # the global map on every rank
        m = res[r][4].reshape(op.n_c, -1)
        assert rel_rms(m[:, op.mask], ref["map"][:, op.mask]) < 1e-5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_one_rank_sharded_solve_equals_plain_solve(precision):
    prob = _problem("Iqu_flags", precision)
    st, it, rel, a1, m1 = _solve_rank(prob, 0, 1, precision,
                                      lambda ptr, count, dtype, stream: 0)
    assert st == ds.DS_OK and rel < 1e-9
    g = prob.to(torch.device("cuda:0"))
    plan = ds.destripe_plan(g.pix, g.c32, g.s32, g.valid, nside=prob.nside, kinds=prob.kinds,
                            baseline_len=prob.baseline_len, precision=precision)
    a = torch.zeros(plan.n_u, dtype=torch.float64, device=g.pix.device)
    st2, _, _ = ds.destripe_solve(plan, g.y, a, tol=1e-10)
    plan.close()
    assert st2 == ds.DS_OK
    assert np.abs(a1.ravel() - a.cpu().numpy()).max() < 1e-5


def test_failing_exchange_ends_the_call():
    prob = _problem("qu", "fp64")
    g = prob.to(torch.device("cuda:0"))
    calls = []

    def bad(ptr, count, dtype, stream):
        calls.append(dtype)
        return 1 if len(calls) > 2 else 0

    plan = ds.destripe_plan_sharded(g.pix, g.c32, g.s32, None, nside=prob.nside,
                                    kinds=prob.kinds, baseline_len=prob.baseline_len,
                                    precision="fp64", allreduce=bad)
    a = torch.zeros(plan.n_u, dtype=torch.float64, device=g.pix.device)
    with pytest.raises(ds.DestripeError) as e:
        ds.destripe_solve_sharded(plan, g.y, a)
    assert e.value.status == ds.DS_ECUDA
    # a sharded plan is refused by the single-domain solve
    with pytest.raises(ds.DestripeError) as e2:
        ds.destripe_solve(plan, g.y, a)
    assert e2.value.status == ds.DS_ESTATE
    plan.close()
