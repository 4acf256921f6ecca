"""The library's schedule (Sec. IV-C/IV-D: Eq. 3-4 weights, the key images, Eq. 5 with the
semi-global half and its seeded slot order, Eq. 8 rates) computed on the host through the C ABI
(gs_schedule_plan, no GPU) against the oracle's restatement, on random overlap graphs -- connected,
partly disconnected, with and without images outside the key set."""
import numpy as np
import pytest

from oracle import schedule as sch


def random_case(rng, n):
    M = rng.uniform(0.0, 1.0, (n, n)).astype(np.float32)
    M = np.triu(M, 1)
    M[rng.uniform(size=M.shape) < 0.5] = 0.0  # sparse overlaps, some images unreachable
    M = (M + M.T).astype(np.float32)
    T = rng.integers(0, 400, n).astype(np.int32)
    return M, T


@pytest.mark.parametrize("seed", range(40))
def test_schedule_plan_matches_the_oracle(seed):
    import paper_2503_13086_gb300 as gs
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 14))
    M, T = random_case(rng, n)
    new = int(rng.integers(0, n))
    T_I, N_m = int(rng.choice([1, 7, 200, 201])), int(rng.integers(1, 11))
    cfg_seed = int(rng.integers(0, 2**63))
    eta0, etaf, T_a = 1.6e-4, 1.6e-6, 200
    got = gs.schedule_plan(M, T, new, T_I=T_I, N_m=N_m, seed=cfg_seed, eta0=eta0, etaf=etaf, T_a=T_a)
    M64 = M.astype(np.float64)
    w, _ = sch.hierarchical_weights(M64, new)
    keys, iters, slots = sch.allocate(w, N_m, T_I, list(range(n)), new, cfg_seed)
    assert got["keys"] == keys
    assert got["slots"] == slots and len(slots) == T_I
    assert np.allclose(got["w"], w, rtol=1e-6, atol=0)
    lr = [sch.lr_image(j, M64, T, T_a, np.float32(eta0), np.float32(etaf)) for j in range(n)]
    assert np.allclose(got["lr"], lr, rtol=1e-6, atol=0)


def test_schedule_plan_rejects_bad_arguments():
    import paper_2503_13086_gb300 as gs
    M = np.zeros((2, 2), np.float32)
    with pytest.raises(gs.GSError):
        gs.schedule_plan(M, [0, 0], 2)
    with pytest.raises(gs.GSError):
        gs.schedule_plan(M, [0, 0], 0, T_I=0)
