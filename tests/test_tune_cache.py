"""The autotuner cache is host state: saved, merged and rejected without a GPU."""
import os

import pytest


def test_tune_cache_round_trip(tmp_path):
    import paper_2410_19075_gb300 as P
    from paper_2410_19075_gb300._lib import SimError
    P.tune_clear()
    f = os.path.join(tmp_path, "tune.txt")
    P.tune_save(f)
    assert [l for l in open(f) if not l.startswith("#")] == []
    with open(f, "a") as fh:
        fh.write("0 1 1000000 350000 2 1\n1 -1 4000 7 1 0\n")
    P.tune_load(f)
    g = os.path.join(tmp_path, "tune2.txt")
    P.tune_save(g)
    assert sorted(l for l in open(g) if not l.startswith("#")) == ["0 1 1000000 350000 2 1\n", "1 -1 4000 7 1 0\n"]
    for bad in ("0 1 5 6 3 1\n", "2 1 5 6 1 0\n", "0 1 5\n", "0 1 5 6 1 2\n"):
        with open(f, "w") as fh:
            fh.write(bad)
        with pytest.raises(SimError):
            P.tune_load(f)
    with pytest.raises(SimError):
        P.tune_load(os.path.join(tmp_path, "missing.txt"))
    P.tune_clear()
