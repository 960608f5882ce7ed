"""LoopConfig: validation of the run knobs and the JSON round trip (host logic, no GPU)."""
import pytest

from paper_2404_17744_gb300.config import LoopConfig


def test_defaults_and_round_trip():
    c = LoopConfig()
    assert (c.precision, c.method, c.mixing, c.tol) == ("fp64", "gf2", "diis", 1e-8)
    d = LoopConfig(precision="bf16x3", method="gwsox", mixing="damp", tol=1e-6, learned_proposals=1,
                   autotune_cache="tiles.txt", checkpoint="loop.npz", metrics="loop.jsonl")
    assert LoopConfig.from_json(d.to_json()) == d


@pytest.mark.parametrize("kw", [dict(precision="tf32"), dict(method="rpa"), dict(mixing="broyden"),
                                dict(damping=0.0), dict(damping=1.5), dict(diis_size=0), dict(diis_size=17),
                                dict(max_iter=0), dict(tol=-1.0), dict(n_damp=-1), dict(learned_proposals=-2)])
def test_bad_values_are_rejected(kw):
    with pytest.raises(ValueError):
        LoopConfig(**kw)
