"""The benchmark's metric against the worked example the thesis prints (Eq. 39), and the
replicas-only multi-process plumbing on CPU (gloo, world size 2)."""
import json
import os

import pytest

from paper_2207_08716_gb300 import measure as M

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "teff_eq39.json")
GOLDEN_41_43 = os.path.join(os.path.dirname(__file__), "golden", "teff_eqs41_43.json")


def test_t_eff_reproduces_eq39():
    g = json.load(open(GOLDEN))
    n = g["n"] ** 3
    kw = dict(unknown=g["unknown_dofs"], known=g["known_dofs"])
    # t_it is printed to 3 significant digits: the printed T_eff lies in the image of that interval
    half = 0.5 * 10 ** (-g["printed_digits"])
    hi = M.t_eff_gbs(n, g["p_bytes"], g["t_it_s"] - half, **kw)
    lo = M.t_eff_gbs(n, g["p_bytes"], g["t_it_s"] + half, **kw)
    assert lo <= g["T_eff_gbs"] <= hi
    assert abs(M.t_eff_gbs(n, g["p_bytes"], g["t_it_s"], **kw) - g["T_eff_gbs"]) < 0.2
    # A_eff = 25 N p (Eq. 37) for the default DOF counts
    assert M.a_eff_bytes(n, 8) == 25 * n * 8


def test_t_eff_reproduces_eqs41_43():
    # the thesis's estimates for three other solvers (Eq. 40 with 12 unknown + 1 known DOF):
    # each printed value is the formula's value rounded to the printed decimals
    for c in json.load(open(GOLDEN_41_43))["cases"]:
        v = M.t_eff_gbs(int(c["N"]), c["p_bytes"], c["t_it_s"])
        assert round(v, c["printed_decimals"]) == c["T_eff_gbs"], (c["eq"], v)


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, lr, w = M.rank_env()
    seed = M.replica_seed(r)
    t = M.max_over_ranks(1.0 + r)              # the slowest rank's time
    tot = M.sum_over_ranks(10.0 * (r + 1))     # units processed by all ranks
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, lr, w, seed, t, tot))


def test_replicas_timing_reduction_gloo_two_ranks():
    import multiprocessing as mp
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[3] for o in out] == [0, 1]          # independent seeds per replica
    assert all(o[4] == 2.0 for o in out)          # max over ranks
    assert all(o[5] == 30.0 for o in out)         # sum over ranks
    assert all(o[2] == 2 for o in out)
