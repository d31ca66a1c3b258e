"""bench.py is only run in full on a GPU; this CPU check catches a name that
no scope of bench.py defines (a missing module-level table or helper) before
a GPU run does."""
import ast
import builtins
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bound(node):
    """Names bound anywhere inside `node` (nested scopes included)."""
    out = set()
    for n in ast.walk(node):
        if isinstance(n, ast.Name) and isinstance(n.ctx, (ast.Store, ast.Del)):
            out.add(n.id)
        elif isinstance(n, (ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)):
            out.add(n.name)
            if not isinstance(n, ast.ClassDef):
                a = n.args
                for arg in a.posonlyargs + a.args + a.kwonlyargs + [a.vararg, a.kwarg]:
                    if arg is not None:
                        out.add(arg.arg)
        elif isinstance(n, ast.Lambda):
            a = n.args
            for arg in a.posonlyargs + a.args + a.kwonlyargs + [a.vararg, a.kwarg]:
                if arg is not None:
                    out.add(arg.arg)
        elif isinstance(n, (ast.Import, ast.ImportFrom)):
            for al in n.names:
                out.add((al.asname or al.name).split(".")[0])
        elif isinstance(n, ast.ExceptHandler) and n.name:
            out.add(n.name)
        elif isinstance(n, (ast.Global, ast.Nonlocal)):
            out.update(n.names)
    return out


def test_every_name_in_bench_is_defined():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    known = _bound(tree) | set(dir(builtins)) | {"__file__", "__name__"}
    missing = sorted({n.id for n in ast.walk(tree)
                      if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load) and n.id not in known})
    assert not missing, f"names used in bench.py but defined nowhere: {missing}"


def test_schedule_parsing_and_traffic_keys():
    """--schedule takes four or five values (the fifth, reference tiles per
    query stage, defaults to one), and every captured DRAM figure is keyed by
    kernel, form and all five schedule values, which is how the bench looks
    it up."""
    import sys
    import pytest
    sys.path.insert(0, ROOT)
    import bench
    assert bench.parse_schedule("16,2,2,2") == {"tile_group": 16, "super_group": 2, "cluster": 2,
                                                "cta_group": 2, "tiles_per_stage": 1}
    assert bench.parse_schedule("8,2,2,2,2")["tiles_per_stage"] == 2
    with pytest.raises(SystemExit):
        bench.parse_schedule("16,2,2")
    assert bench.TRAFFIC
    for key, v in bench.TRAFFIC.items():
        assert len(key) == 2 + len(bench.SCHEDULE_KEYS) and key[0].startswith("k_search")
        assert v["bytes"] > 0 and len(v["sha256"]) == 16
    # the default schedule and every kind::mxf4 candidate of the autotuner's grid resolve to a figure
    for tg in (4, 8, 16, 32):
        for sg in (2, 4, 16):
            for tps in (1, 2):
                assert ("k_search_mma2", "tc_mxf4", tg, sg, 2, 2, tps) in bench.TRAFFIC
