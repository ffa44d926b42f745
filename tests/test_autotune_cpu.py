"""Host logic of the autotuner and the benchmark's bookkeeping, on CPU:
Sec. 5.2's break-even solve count, the tuning cache of ``bench.py
--tune-cache``, the autotuner's staged search over forms and launch shapes
(against a plan whose solve times follow a fixed model), and the tuning row
the benchmark prints for the partitioned form."""

import torch


def test_break_even_solve_count():
    """Sec. 5.2's n_s: the smallest number of solves after which a costlier
    setup with faster solves has the shorter total time."""
    import bench
    assert bench._break_even(10.0, 1.0, 5.0, 2.0) == 6      # 16 < 17, but 15 == 15
    assert bench._break_even(4.0, 1.0, 5.0, 2.0) == 0       # cheaper setup and faster solves
    assert bench._break_even(10.0, 3.0, 5.0, 2.0) is None   # never
    for sa, ta, sb, tb in ((29.0, 0.5, 11.0, 1.0), (57.0, 0.66, 102.0, 2.05)):
        k = bench._break_even(sa, ta, sb, tb)
        assert sa + k * ta < sb + k * tb
        assert k == 0 or not (sa + (k - 1) * ta < sb + (k - 1) * tb)


class _FakePlan:
    """Records the tuning calls the autotuner makes (no GPU)."""

    def __init__(self):
        self.calls = []
        self.best_algo = "self"

    def set_tuning(self, lanes, block, max_blocks):
        self.calls.append(("tuning", lanes, block, max_blocks))

    def set_tiling(self, tile_rows, level_order=False):
        self.calls.append(("tiling", tile_rows, level_order))

    def set_partition(self, part_rows=0, cluster_blocks=1):
        self.calls.append(("partition", part_rows, cluster_blocks))


def test_tune_cache_round_trip():
    """The benchmark's tune cache stores the autotuner's choice as JSON and
    re-applies it without timing anything (a profiler run of the same command
    then uses the plain run's launch shapes)."""
    import json

    from paper_1710_04985_gb300 import autotune
    for algo, tiles in (("permuted", False), ("blocked", True), ("tiled", True)):
        result = {"algo": algo, "best": (2, 128, 608, 0.47, 512, False), "per_algo": {}}
        ch = json.loads(json.dumps(autotune.choice(result)))
        assert ch == [algo, 2, 128, 608, 512, False]
        p = _FakePlan()
        out = autotune.apply_choice(p, ch)
        assert p.best_algo == algo and out["algo"] == algo
        assert p.calls[0] == ("tuning", 2, 128, 608)
        assert (("tiling", 512, False) in p.calls) == tiles
    # the partitioned form: part rows and thread-block cluster size
    result = {"algo": "partitioned", "best": (1, 512, 0, 0.44, 16384, 4), "per_algo": {}}
    ch = json.loads(json.dumps(autotune.choice(result)))
    assert ch == ["partitioned", 1, 512, 0, 16384, 4]
    p = _FakePlan()
    autotune.apply_choice(p, ch)
    assert p.calls == [("tuning", 1, 512, 0), ("partition", 16384, 4)]
    p = _FakePlan()
    autotune.apply_choice(p, ["partitioned", 1, 512, 0, 0, False])   # no cluster recorded
    assert p.calls[-1] == ("partition", 0, 1)


class _ModelPlan(_FakePlan):
    """A plan whose solve time is a fixed function of its launch shape, for
    checking the autotuner's search and bookkeeping without a GPU."""

    class _Ptr:
        def __init__(self, v):
            self.v = v

        def data_ptr(self):
            return self.v

    def __init__(self):
        super().__init__()
        import torch
        self.n, self.nnz, self.upper, self.unit, self.dtype = 1000, 4000, False, False, torch.float64
        self.rowptr, self.colidx = self._Ptr(1), self._Ptr(2)
        self.shape = (4, 256, 0)
        self.part = (0, 1)
        self.algo_shapes = {}

    def set_tuning(self, lanes, block, max_blocks):
        super().set_tuning(lanes, block, max_blocks)
        self.shape = (lanes, block, max_blocks)
        self.algo_shapes = {}

    def set_partition(self, part_rows=0, cluster_blocks=1):
        super().set_partition(part_rows, cluster_blocks)
        self.part = (part_rows, cluster_blocks)

    def set_algo_tuning(self, algo, lanes, block, max_blocks):
        self.algo_shapes[algo] = (lanes, block, max_blocks)

    def model_ms(self, algo):
        lanes, block, _ = self.shape
        base = {"self": 1.0, "permuted": 0.9, "partitioned": 0.8}.get(algo, 2.0)
        if algo == "partitioned":
            rows, cl = self.part
            base += (0.0 if rows == 16384 else 0.1) - (0.05 if cl == 4 else 0.0)
            return base + (0.0 if lanes == 1 else 0.2) + (0.0 if block == 512 else 0.03)
        return base + (0.0 if lanes == 2 else 0.2) + (0.0 if block == 128 else 0.03)


def test_autotuner_search_and_per_form_shapes(monkeypatch):
    """tune_algos keeps the fastest form, applies its shape (for the
    partitioned form: part size and cluster size too), and records every
    measured form's own best shape on the plan."""
    import types

    import torch

    from paper_1710_04985_gb300 import autotune
    monkeypatch.setattr(torch.cuda, "get_device_properties",
                        lambda dev: types.SimpleNamespace(multi_processor_count=152))
    monkeypatch.setattr(autotune, "time_solve",
                        lambda plan, b, x, algo="self", reps=3, transpose=False:
                        plan.model_ms(algo))
    p = _ModelPlan()
    b = torch.zeros(1000, dtype=torch.float64)
    res = autotune.tune_algos(p, b, torch.empty_like(b), use_cache=False,
                              algos=("self", "permuted", "partitioned"))
    assert res["algo"] == "partitioned" and p.best_algo == "partitioned"
    lanes, block, max_blocks, ms, rows, cluster = res["best"]
    assert (lanes, block, rows, cluster) == (1, 512, 16384, 4)
    assert abs(ms - 0.75) < 1e-12
    assert p.part == (16384, 4)
    # every form keeps its own best shape; the in-place and level-ordered forms
    # prefer 2 lanes and 128 threads in this model
    assert p.algo_shapes["partitioned"][:2] == (1, 512)
    assert p.algo_shapes["self"][:2] == (2, 128)
    assert p.algo_shapes["permuted"][:2] == (2, 128)
    # the cluster stage ran for the partitioned form only
    assert ("partition", 16384, 2) in p.calls and ("partition", 16384, 4) in p.calls


def test_bench_tuning_row_reports_parts_and_clusters():
    import bench
    assert bench._tuning_row({"algo": "partitioned", "best": (1, 512, 0, 0.4, 16384, 4)}) == \
        [1, 512, 0, 16384, 4]
    assert bench._tuning_row({"algo": "partitioned", "best": (1, 512, 0, 0.4, 0, False)}) == \
        [1, 512, 0, 0, 1]
    assert bench._tuning_row({"algo": "tiled", "best": (4, 256, 0, 0.4, 2048, True)}) == \
        [4, 256, 0, 2048, True]
    assert bench._tuning_row({"algo": "permuted", "best": (2, 128, 608, 0.4, 2048, False)}) == \
        [2, 128, 608, None, None]


class _InteractingPlan(_ModelPlan):
    """A plan whose best width depends on the block size (as on the
    512-system batch: 8 lanes win at 512 threads, 16 lanes at 1024 win
    overall)."""

    def model_ms(self, algo):
        lanes, block, _ = self.shape
        table = {(8, 512): 6.0, (16, 512): 6.4, (8, 1024): 5.4, (16, 1024): 4.7}
        return table.get((lanes, block), 9.0)


def test_autotuner_searches_width_and_block_together(monkeypatch):
    """For the tiled forms with two block sizes or fewer the first stage runs
    every width at every block size, so a width that only wins at the larger
    block is found."""
    import types

    import torch

    from paper_1710_04985_gb300 import autotune
    monkeypatch.setattr(torch.cuda, "get_device_properties",
                        lambda dev: types.SimpleNamespace(multi_processor_count=152))
    monkeypatch.setattr(autotune, "time_solve",
                        lambda plan, b, x, algo="self", reps=3, transpose=False:
                        plan.model_ms(algo))
    p = _InteractingPlan()
    b = torch.zeros(1000, dtype=torch.float64)
    res = autotune.tune(p, b, torch.empty_like(b), algo="partitioned", use_cache=False,
                        **autotune.QUICK["partitioned"])
    lanes, block = res["best"][:2]
    assert (lanes, block) == (16, 1024) and abs(res["best"][3] - 4.7) < 1e-12
    tried = {(r[0], r[1]) for r in res["table"]}
    assert {(8, 512), (8, 1024), (16, 512), (16, 1024)} <= tried
