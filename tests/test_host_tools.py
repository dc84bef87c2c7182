"""CPU tests of the host-side tools around the library: the autotuner's cache, the
serving mix, and the bench's choice of kernel label (no GPU needed)."""
import numpy as np

import workloads


def test_autotune_cache_round_trip(tmp_path, monkeypatch):
    from paper_2211_17263_gb300 import autotune
    path = str(tmp_path / "sub" / "tune.json")
    monkeypatch.setenv("PRDPT_AUTOTUNE_CACHE", path)
    assert autotune.default_cache() == path
    wl = workloads.scaled(workloads.config_caustic(), width=40, height=32, spp=4, pairs=4)
    assert autotune.cached_shape(wl) is None  # no file yet
    entry = {"block_pixels": 16, "ctas_per_sm": 2, "render_groups": 0, "no_path_sharing": 0, "ms": 1.5}
    autotune._store(path, {autotune.shape_key(wl): entry})
    hit = autotune.cached_shape(wl)
    assert hit is not None and hit["block_pixels"] == 16 and hit["ctas_per_sm"] == 2
    assert autotune.cached_shape(wl, None) is None  # lookups disabled
    # another shape (more renders) misses; a corrupt file reads as empty
    other = workloads.scaled(wl, pairs=8)
    assert autotune.shape_key(other) != autotune.shape_key(wl) and autotune.cached_shape(other) is None
    with open(path, "w") as f:
        f.write("{not json")
    assert autotune.cached_shape(wl) is None


def test_autotune_candidates_cover_every_knob():
    from paper_2211_17263_gb300.autotune import CANDIDATES
    assert len(CANDIDATES) == len(set(CANDIDATES)) == 18
    assert {c[0] for c in CANDIDATES} == {8, 16, 32}
    assert {c[1] for c in CANDIDATES} == {2, 3}
    assert {(c[2], c[3]) for c in CANDIDATES} == {(0, 0), (-1, 0), (0, 1)}


def test_serving_mix_is_seeded_and_follows_its_recipe():
    a = workloads.serving_mix(64, seed=3, rate_hz=0.5)
    b = workloads.serving_mix(64, seed=3, rate_hz=0.5)
    assert [w.name for _, w in a] == [w.name for _, w in b]
    assert [t for t, _ in a] == [t for t, _ in b]
    times = [t for t, _ in a]
    assert times == sorted(times) and times[0] > 0.0
    kinds = set()
    for _, wl in a:
        assert wl.width == wl.height and wl.width in range(128, 513, 64)
        assert wl.renders in (8, 16, 32, 64) and wl.spp in (8, 16, 32, 64)
        kind = wl.name.split("-")[1]
        kinds.add(kind)
        assert wl.steps == (300 if kind == "gi" else 100)
        assert np.all(np.isfinite(wl.theta_ref)) and np.all(np.isfinite(wl.theta0))
    assert kinds == {"small", "occlusion", "gi"}
    assert [w.name for _, w in workloads.serving_mix(8, seed=4)] != [w.name for _, w in a[:8]]


def test_bench_labels_emitter_jobs():
    import bench
    assert bench._emitter_bound(workloads.config_caustic())      # the light moves
    assert bench._emitter_bound(workloads.config_gi_box())       # the light moves (beside albedos)
    assert not bench._emitter_bound(workloads.config_occlusion())  # a box moves
    assert not bench._emitter_bound(workloads.config_small())      # a sphere moves


def test_bench_profile_values_parse(tmp_path, monkeypatch):
    """A profile summary's machine-readable lines are read only while its kernel source
    hash matches the current sources."""
    import bench
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_kernel_source_sha", lambda read=None: "abc123")
    body = "- kernel_source_sha: `{}`\n- dram_bytes_per_step: `1234`\n- fp32_flop_per_step: `5e9`\n"
    (prof / "render_pipeline_w_ncu.md").write_text(body.format("abc123"))
    assert bench._profiled("w", "dram_bytes_per_step") == 1234.0
    assert bench._profiled("w", "fp32_flop_per_step") == 5e9
    assert bench._profiled("w", "warp_instructions_per_step") is None
    (prof / "render_pipeline_w_ncu.md").write_text(body.format("other"))
    assert bench._profiled("w", "dram_bytes_per_step") is None
    assert bench._profiled("missing", "dram_bytes_per_step") is None


def test_bench_launch_count_per_step():
    """Launches per resident step by job kind (the launch lists in profiles/ show the same)."""
    import bench
    assert bench._launches_per_step(workloads.config_caustic(), sharing=True) == 3  # emitter sharing
    assert bench._launches_per_step(workloads.config_occlusion(), sharing=True) == 5  # path sharing
    assert bench._launches_per_step(workloads.config_gi_box(), sharing=False) == 3  # render groups
    assert bench._launches_per_step(workloads.config_texture(), sharing=False) == 6  # + draws, norms, gradient
