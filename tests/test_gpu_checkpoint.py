"""Checkpoint and resume: a run saved at step 11 and resumed in a new Simulation (lbm_attach
on the saved state bytes) reaches step 23 with the same fields, bit for bit, as a run that
never stopped; for the fused two-buffer flow layout (odd time level: the state lives in the
second copy) and for the in-place AA layout without flow."""
import pytest
import torch

from workloads import configs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["flow", "ripening"])
def test_resume_is_bit_identical(case, tmp_path):
    from paper_2409_03401_gb300 import Simulation
    if case == "flow":
        p, fields = configs.sedimentation(shape=(20, 24, 40), fraction=0.05, r=(3.0, 5.0))
    else:
        p, fields = configs.ripening(shape=(16, 18, 40))
    f = [t.cuda() for t in fields()]
    ref = Simulation(p, *f)
    ref.step(23)
    a = Simulation(p, *f)
    a.step(11)
    path = tmp_path / "ck.pt"
    a.save(path)
    del a
    b = Simulation.load(path)
    assert b.t == 11
    b.step(12)
    torch.cuda.synchronize()
    assert b.t == ref.t == 23
    # every field of the time level, bit for bit (the raw state also holds plane padding
    # that no kernel writes, so it is not compared byte for byte)
    fr, fb = ref.fields(), b.fields()
    for k in fr:
        assert torch.equal(fr[k], fb[k]), k
