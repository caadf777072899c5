"""rick_predict (model visibilities from a model image, by degridding) against
the FP64 oracle's prediction on the same inputs: max |V_gpu - V_oracle| <=
1e-4 max |V_oracle|.  With grid correction the model is divided by c(x) c(y)
(up to ~1e4 at the corners of the KB support-7 taper), which amplifies FP32
rounding; the random models are therefore weighted by c(x) c(y), as the
adjoint's dot-product tests weight their images (the division itself is
still applied)."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

KB = synth.KERNEL_KB
CORRECT, REAL, APPLY_N, FOLD = synth.FLAG_CORRECT, synth.FLAG_REAL, synth.FLAG_APPLY_N, synth.FLAG_FOLD


@pytest.fixture(scope="module")
def rick():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_00959_gb300 import build
    build.build()
    import paper_2504_00959_gb300 as r
    r.load()
    return r


@pytest.mark.parametrize("flags,extra", [(CORRECT | REAL, {}), (CORRECT, {}), (REAL | APPLY_N, {"plane_group": 3}),
                                         (CORRECT | REAL | FOLD, {"w_min": 0.0, "nw": 4}),
                                         (CORRECT | REAL, {"tile": 16})])
def test_predict_matches_oracle(rick, oracle_mod, flags, extra):
    prob = synth.disk_problem(128, 7, 30000, KB, 7, 6.0, 120.0, 301, fill=0.42)
    params = dict(prob["params"], **extra)
    n = params["n"]
    rng = np.random.default_rng(9)
    model = rng.standard_normal((n, n))
    if not flags & REAL:
        model = model + 1j * rng.standard_normal((n, n))
    if flags & CORRECT:
        c = oracle_mod.taper(n, params["kernel"], params["support"], 0.0)
        model = model * np.outer(c, c)
    im = rick.Imager(dict(params, flags=flags))
    g = {k: prob[k].cuda() for k in ("u", "v", "w")}
    dev_model = torch.from_numpy(model.astype(np.float32 if flags & REAL else np.complex64)).cuda()
    got = im.predict(dev_model, g["u"], g["v"], g["w"]).cpu().numpy()
    im.close()
    p = synth.to_numpy(prob)
    ref = oracle_mod.predict(params, p["u"], p["v"], p["w"], model.astype(np.complex128), flags=flags & ~REAL)
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))


def test_predict_point_source_at_the_centre(rick):
    """A unit pixel at the phase centre predicts V = 1 for every measurement
    (the measurement equation at l = m = 0, n = 1), to FP32 rounding."""
    prob = synth.disk_problem(256, 8, 20000, KB, 7, 3.0, 60.0, 303, fill=0.42)
    n = 256
    model = torch.zeros((n, n), device="cuda")
    model[n // 2, n // 2] = 1.0
    im = rick.Imager(dict(prob["params"], flags=CORRECT | REAL))
    got = im.predict(model, prob["u"].cuda(), prob["v"].cuda(), prob["w"].cuda()).cpu().numpy()
    im.close()
    assert np.max(np.abs(got - 1.0)) <= 1e-5


def test_predict_needs_no_forward_pass_and_refuses_batches(rick):
    prob = synth.config1()
    im = rick.Imager(dict(prob["params"], flags=REAL))
    v = im.predict(torch.zeros((256, 256), device="cuda"), prob["u"].cuda(), prob["v"].cuda(), prob["w"].cuda())
    assert torch.count_nonzero(v).item() == 0
    im.close()
    bi = rick.BatchImager(dict(prob["params"], flags=REAL), [(-50.0, 50.0), (-40.0, 40.0)])
    with pytest.raises(rick.RickError):
        bi.predict(torch.zeros((256, 256), device="cuda"), prob["u"].cuda(), prob["v"].cuda(), prob["w"].cuda())
    bi.close()
