"""The autotuner's cache file (no GPU): "key value" lines are merged into the process-wide
cache and read back by key; a missing key reads as absent."""
import os


def test_cache_file_round_trip(tmp_path):
    from paper_2101_01231_gb300 import ridg as R
    p = tmp_path / "tune.txt"
    p.write_text("corr3.block nb3 S4 256\ngemm3.slots nb3 S4 box8 6\nnot a pair\n")
    assert R.ridg_tune_load(str(p)) == R.RIDG_OK
    assert R.ridg_tune_lookup("corr3.block nb3 S4") == 256
    assert R.ridg_tune_lookup("gemm3.slots nb3 S4 box8") == 6
    assert R.ridg_tune_lookup("newton.grid nb9 m1 flux1 prec3") is None
    with __import__("pytest").raises(R.RidgError):
        R.ridg_tune_load(os.path.join(str(tmp_path), "missing.txt"))
