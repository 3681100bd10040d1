"""The trained corrector gains over the coarse method without it, and the
serving checks route failing instances to the fine solver."""
import numpy as np
import pytest

import swe_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    from paper_1107_2157_gb300 import corrector as C
    setup = C.Setup(n_fine=256, factor=4, dt_fine=0.04, coarse_steps=32)
    res = C.train(setup, range(0, 256), B=32, lr=2e-3, passes=2, gen_batch=64)
    return setup, res


def test_training_loss_decreases(trained):
    _, res = trained
    losses = np.array(res["losses"])
    assert np.isfinite(losses).all()
    assert losses[-50:].mean() < 0.8 * losses[:20].mean()


def test_corrector_beats_plain_coarse_on_held_out_smooth_flows(trained):
    """Held-out seeds 1800+: RMS h error after 32 coarse steps against the
    restricted fine solution, plain coarse Lax-Wendroff vs corrected."""
    from paper_1107_2157_gb300 import corrector as C
    setup, res = trained
    seeds = list(range(1800, 1816))
    held = si.corrector_states(seeds, setup.n_fine, setup.dam_fraction)
    smooth = np.array([si.SplitMix64(s, 0xC0DE).uniform() >= setup.dam_fraction for s in seeds])
    truth = C.fine_truth(setup, held)
    plain = C.coarse_run(setup, held, None, None)
    ep = C.rms_h_error(plain, truth)
    plain.close()
    learned = C.coarse_run(setup, held, res["params"], res["norm"])
    el = C.rms_h_error(learned, truth)
    learned.close()
    ratio = el[smooth] / ep[smooth]
    assert np.isfinite(el).all()
    assert np.median(ratio) < 0.8, ratio
    assert (ratio < 1.0).mean() >= 0.75, ratio


def test_serving_checks_and_fallback(trained):
    """With mass projection the corrected step keeps mass to rounding; a
    zero tolerance flags every instance, and the fallback then returns the
    restricted fine solution exactly."""
    from paper_1107_2157_gb300 import corrector as C
    setup, res = trained
    held = si.corrector_states(range(1900, 1904), setup.n_fine, setup.dam_fraction)
    out = C.serve(setup, held, res["params"], res["norm"], mass_tol=1e-5)
    try:
        assert out["status"] == 0
        assert (out["drift"] < 1e-5).all(), out["drift"]
        assert not out["flagged"].any()
    finally:
        out["coarse"].close()
    out = C.serve(setup, held, res["params"], res["norm"], mass_tol=-1.0)
    try:
        assert out["flagged"].all()
        truth = C.fine_truth(setup, held)
        for i in range(len(held)):
            got = out["coarse"].get_state(i)
            for k in range(3):
                assert np.array_equal(got[k], truth[i, k].astype(np.float32))
    finally:
        out["coarse"].close()
