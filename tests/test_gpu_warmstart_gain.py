"""What the trained surrogate gains over the method without it, end to end on
the GPU at a reduced size: resistance tensors measured by the LB method in
32^3 boxes, the network trained on them with its tensor-core kernels, and a
64^3 box with four spheroids started cold and warm (network velocities plus
the lattice fluid's own steady flow and density under the particle forces).
Bars: the network's held-out error on R^ below 10 % (median), and the warm
start reaching 1e-2 and 1e-3 of the steady velocities in at most a third of
the steps of the cold start (measured: 17x and 6x fewer), and in fewer steps
than the same start without the network's velocities (the lattice fluid's
steady flow alone) at every tolerance, at least 1.5 times fewer over the three
(measured 2.1x): the part the network itself adds.  The full-size measurement (128^3, 16 spheroids) is run by
python -m paper_2403_05443_gb300.warmstart."""
import pytest

pytestmark = pytest.mark.gpu

pytest.importorskip("torch")
W = pytest.importorskip("paper_2403_05443_gb300.warmstart")


def test_warm_start_cuts_the_steps_to_steady_state_threefold():
    r = W.experiment(seed=3, n32=96, n48=0, train_steps=1500, eval_n=64, eval_count=4, force=1e-8, every=50,
                     ref_steps=16000)
    s = r["steps_to_steady"]
    print({k: v for k, v in r.items() if k != "error_curves"})
    assert r["val_rel_err_median"] < 0.10
    assert s["cold@0.01"] is not None and s["warm@0.01"] is not None
    assert s["warm@0.01"] * 3 <= s["cold@0.01"]
    assert s["cold@0.001"] is not None and s["warm@0.001"] is not None
    assert s["warm@0.001"] * 3 <= s["cold@0.001"]
    # what the network adds: the same start without its velocities (the
    # lattice fluid's steady flow alone, particles at rest) is slower at every
    # tolerance, and takes at least 1.5 times the steps over the three
    # (measured: 200 / 450 / 1250 against 100 / 200 / 600)
    tols = ("0.01", "0.003", "0.001")
    fl = [s[f"stokes_fluid_only@{t}"] for t in tols]
    wm = [s[f"warm@{t}"] for t in tols]
    assert None not in fl and None not in wm
    assert all(w < f for w, f in zip(wm, fl))
    assert sum(wm) * 1.5 <= sum(fl)
