"""Guard words behind every device buffer (debug_canaries): a session's kernels never write past a
buffer's end -- single- and multi-view steps, the field update, densification, snapshot / restore
-- and a guard changed on the host (as a kernel writing past the end would) is reported, naming
the buffer."""
import numpy as np
import pytest

import gsinputs as gi

pytestmark = pytest.mark.gpu


def session(debug=1, seed=3):
    import paper_2503_13086_gb300 as gs
    p = gi.cube_scene(3000, seed=seed, stride=3000)
    f = gs.Field(scene_extent=1.0, tiling=(16, 16, 256), use_graph=1, seed=seed, debug_canaries=debug,
                 densify_stats=1)
    f.set_gaussians(p)
    cams = [gi.identity_camera(96, 64, 90.0), gi.identity_camera(70, 52, 60.0)]
    R, t = gi.look_at([0.4, -0.3, -0.4], [0.0, 0.0, 3.0])
    cams.append(gi.camera_dict(R, t, 70.0, 70.0, 40.0, 30.0, 81, 61))
    ids = [f.add_image(c, gi.uniform_target(c["width"], c["height"], 30 + k)) for k, c in enumerate(cams)]
    return f, ids


def test_guards_stay_intact_through_a_session():
    import paper_2503_13086_gb300 as gs
    f, ids = session()
    for k in range(3):
        f.optimize_step([ids[k]])
    f.optimize_step(ids)
    f.snapshot()
    f.optimize_step(ids[:2])
    f.restore()
    f.densify(grad_thresh=1e-7, percent_dense=0.02, min_opacity=0.01, max_scale=0.5)
    for _ in range(2):
        f.optimize_step(ids)
    assert np.isfinite(f.optimize_step([ids[0]]))
    f.close()


@pytest.mark.parametrize("which", [0, 1, 2])
def test_a_changed_guard_is_reported_with_the_buffer_name(which):
    import paper_2503_13086_gb300 as gs
    f, ids = session()
    f.optimize_step(ids)
    # the first allocated buffer, one in the middle and the last one (an index out of range names
    # the valid ones)
    with pytest.raises(gs.GSError) as e:
        f.corrupt_guard(10_000)
    n = int(str(e.value).rsplit("..", 1)[1]) + 1
    assert n > 30
    index = [0, n // 2, n - 1][which]
    name = f.corrupt_guard(index)
    with pytest.raises(gs.GSError) as e:
        f.optimize_step([ids[0]])
    assert e.value.status == 9 and f"'{name}'" in str(e.value)
    f.close()


def test_without_the_check_a_changed_guard_goes_unnoticed():
    f, ids = session(debug=0)
    f.optimize_step(ids)
    f.corrupt_guard(0)
    assert np.isfinite(f.optimize_step(ids))
    f.close()
