"""Failure detection without a GPU fault: the bounded inter-CTA waits of the scan (K2) and of the
sort passes (K4), and the loss forward's waits for the blend forward's tile flags and warp count.
Each wait runs once with a predecessor that never starts (or a flag nothing sets), so it can only end
by giving up; it must report that through the control block, return, and leave the context usable
for the next step."""
import numpy as np
import pytest

import gsinputs as gi

pytestmark = pytest.mark.gpu


def small_step(seed=4):
    import paper_2503_13086_gb300 as gs
    p = gi.cube_scene(2000, seed=seed, stride=2000)
    cam = gi.identity_camera(96, 64, 90.0)
    f = gs.Field(scene_extent=1.0, tiling=(16, 16, 256), use_graph=0, seed=seed)
    f.set_gaussians(p)
    img = f.add_image(cam, gi.uniform_target(96, 64, seed))
    loss = f.optimize_step([img])
    out = f.get_gaussians(with_adam=True)
    f.close()
    return loss, out


def test_both_waits_give_up_and_report_it():
    import paper_2503_13086_gb300 as gs
    (e_scan, e_sort), (ms_scan, ms_sort) = gs.wait_probe(spin_limit=4096)
    assert e_scan & 1, "the scan's look-back did not report giving up"
    assert e_sort & 1, "the sort pass's look-back did not report giving up"
    assert 0.0 < ms_scan < 1000.0 and 0.0 < ms_sort < 1000.0


def test_the_wait_is_bounded_by_its_limit():
    import paper_2503_13086_gb300 as gs
    (_, _), (a_scan, a_sort) = gs.wait_probe(spin_limit=1 << 10)
    (_, _), (b_scan, b_sort) = gs.wait_probe(spin_limit=1 << 14)
    # sixteen times the rounds take several times as long (the wait spins; it does not block)
    assert b_scan > 4.0 * a_scan and b_sort > 4.0 * a_sort


def test_the_context_stays_usable_after_a_wait_gave_up():
    import paper_2503_13086_gb300 as gs
    before = small_step()
    (e_scan, e_sort), _ = gs.wait_probe(spin_limit=2048)
    assert e_scan & 1 and e_sort & 1
    after = small_step()
    assert before[0] == after[0]
    for a, b in zip(before[1], after[1]):
        assert np.array_equal(a, b)


def test_the_steps_own_limit_gives_up_within_a_few_seconds():
    import paper_2503_13086_gb300 as gs
    (e_scan, e_sort), (ms_scan, ms_sort) = gs.wait_probe(spin_limit=0)
    assert e_scan & 1 and e_sort & 1
    assert 100.0 < ms_scan < 5000.0 and 100.0 < ms_sort < 5000.0


def test_the_loss_waits_give_up_and_report_it():
    import paper_2503_13086_gb300 as gs
    err, ms = gs.loss_wait_probe(spin_limit=4096)
    assert err & 1, "the loss forward's waits did not report giving up"
    assert 0.0 < ms < 1000.0


def test_the_loss_waits_are_bounded_by_their_limit():
    import paper_2503_13086_gb300 as gs
    _, a = gs.loss_wait_probe(spin_limit=1 << 10)
    _, b = gs.loss_wait_probe(spin_limit=1 << 14)
    assert b > 4.0 * a


def test_the_context_stays_usable_after_the_loss_waits_gave_up():
    import paper_2503_13086_gb300 as gs
    before = small_step()
    err, _ = gs.loss_wait_probe(spin_limit=2048)
    assert err & 1
    after = small_step()
    assert before[0] == after[0]
    for a, b in zip(before[1], after[1]):
        assert np.array_equal(a, b)


def test_the_steps_own_loss_wait_limit_gives_up_within_seconds():
    import paper_2503_13086_gb300 as gs
    err, ms = gs.loss_wait_probe(spin_limit=0)
    assert err & 1
    assert 100.0 < ms < 10000.0
