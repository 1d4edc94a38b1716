"""Host logic of the autotuner: candidate set, choice of the fastest, cache round trip (no GPU)."""
from paper_2509_23945_gb300 import autotune, tnmc


class FakeContext:
    def __init__(self, precision):
        self.precision = precision
        self.workloads = [None]
        self.applied = []

    def set_tuning(self, **cfg):
        self.applied.append(dict(cfg))


def test_candidates_cover_the_result_preserving_choices():
    keep = autotune.candidates(tnmc.PREC_F32)
    assert len(keep) == 12 and {c["gemm_mode"] for c in keep} == {-1}      # engine untouched by default
    assert {c["gemm_tile"] for c in keep} == {0, 1, 2}
    f32 = autotune.candidates(tnmc.PREC_F32, allow_arith_changes=True)
    assert len(f32) == 24 and {c["gemm_mode"] for c in f32} == {0, 1}
    assert {(c["eig_smem"], c["ctas_per_sm"]) for c in f32} == {(1, 2), (1, 1), (0, 2), (0, 1)}
    f64 = autotune.candidates(tnmc.PREC_F64)
    assert len(f64) == 4 and all(c["gemm_mode"] == -1 and c["gemm_tile"] == -1 for c in f64)
    assert all("jac_floor" not in c for c in f32 + f64)      # changes results: never tuned


def test_tune_applies_the_fastest_and_caches_it(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(autotune, "_key", lambda ctx, group, prec: f"gpu|prec={prec}")
    # seconds per slice: fastest is gemm 0, eig in shared memory, 2 CTAs per SM
    cost = lambda c: (1.0 + 0.5 * c["gemm_mode"] + 0.25 * (1 - c["eig_smem"]) + 0.125 * (2 - c["ctas_per_sm"])
                      + 0.0625 * abs(c["gemm_tile"] - 2))
    ctx = FakeContext(tnmc.PREC_F32)
    monkeypatch.setattr(autotune, "time_config", lambda ctx, group, n: cost(ctx.applied[-1]))
    out = autotune.tune(ctx, group=0, n_chains=4, allow_arith_changes=True)
    assert out["best"] == dict(gemm_mode=0, eig_smem=1, ctas_per_sm=2, gemm_tile=2)
    assert ctx.applied[-1] == out["best"]
    times = [t["s_per_slice"] for t in out["times"]]
    assert times == sorted(times) and len(times) == 24
    fresh = FakeContext(tnmc.PREC_F32)
    assert autotune.apply_cached(fresh, group=0) == out["best"]
    assert fresh.applied == [out["best"]]
    assert autotune.apply_cached(FakeContext(tnmc.PREC_F64), group=0) is None
