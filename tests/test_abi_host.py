"""Host-side checks of the C ABI boundary (no GPU needed).

* the compiled library exports every function ``include/idw.h`` declares;
* the launch plan's stream-K split covers every work unit exactly once and
  gives every (query tile, CTA) piece a distinct partial slot;
* ceiling-division split arithmetic, pinned to the paper's worked example
  (Sec. 3.1: 3000 points over 1024 threads -> 3 per thread);
* argument errors surface as status codes / exceptions, not crashes.
"""
import ctypes
import json
import os
import re

import numpy as np
import pytest

from paper_1402_4986_gb300 import build as idw_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    idw_build.build()
    from paper_1402_4986_gb300 import _lib
    return _lib.load()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "idw.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(idw_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("idw_create", "idw_destroy", "idw_interpolate", "idw_interpolate_batched",
                     "idw_backward", "idw_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1402_4986_gb300 import _lib
    for name in _declared_functions():
        assert hasattr(lib, name), f"{name} not exported"
        assert name in _lib.SIGNATURES, f"{name} has no ctypes signature in the binding"


def test_binding_options_match_the_header():
    """Every idw_option of the header has the binding's name and value, and
    the binding names no option the header lacks."""
    text = open(os.path.join(ROOT, "include", "idw.h")).read()
    declared = {m.group(1).lower(): int(m.group(2))
                for m in re.finditer(r"\bIDW_OPT_([A-Z0-9_]+)\s*=\s*(\d+)", text)}
    from paper_1402_4986_gb300 import _lib
    assert declared == _lib.OPTIONS


def test_status_strings(lib):
    for code, name in {0: "IDW_OK", 1: "IDW_ERR_INVALID_ARG", 7: "IDW_ERR_DEVICE_TIMEOUT"}.items():
        assert lib.idw_status_string(code).decode() == name


def test_null_handle_is_rejected(lib):
    assert lib.idw_interpolate(None, None, 10, None, 10, 2.0, 0, None, None) == 1
    assert lib.idw_destroy(None) == 1
    assert lib.idw_sync_status(None, None) == 1
    assert lib.idw_interpolate_local(None, None, 10, None, 10, 2.0, 0.1, None, None, None) == 1
    assert lib.idw_interpolate_knn(None, None, 10, None, 10, 2.0, 4, None, None, None, None) == 1
    ix = ctypes.c_void_p()
    assert lib.idw_local_index_create(None, None, 10, 0.1, 0, ctypes.byref(ix), None) == 1
    assert not ix.value
    assert lib.idw_local_index_interpolate(None, None, None, 10, 2.0, 0.1, None, None, None) == 1
    assert lib.idw_local_index_knn(None, None, None, 10, 2.0, 4, None, None, None, None) == 1
    assert lib.idw_local_index_destroy(None) == 1
    assert lib.idw_local_index_modified(None, None, None, 10, 2.0, 0.1, None, None, None) == 1
    assert lib.idw_interpolate_modified(None, None, 10, None, 10, 2.0, 0.1, None, None, None) == 1
    for fn in (lib.idw_local_backward, lib.idw_modified_backward):
        assert fn(None, None, 10, None, 10, 2.0, 0.1, None, None, None, None, None, None) == 1
    assert lib.idw_knn_backward(None, None, 10, None, 10, 2.0, 4, None, None, None, None, None,
                                None) == 1
    out = ctypes.c_void_p()
    assert lib.idw_create(None, 0) == 1


def _cover(plan):
    """Replays the stream-K split on the host: unit -> CTA and piece slots."""
    U, G, Td = plan["units"], plan["grid"], plan["data_tiles"]
    begins = [g * U // G for g in range(G + 1)]
    owner = np.empty(U, np.int64)
    slots = set()
    for g in range(G):
        owner[begins[g]:begins[g + 1]] = g
        for u in range(begins[g], begins[g + 1]):
            slots.add((u // Td) + g)
    return owner, slots


@pytest.mark.parametrize("n,m,sms,ctas", [
    (1, 1, 152, 2), (255, 3, 152, 2), (256, 2048, 152, 2), (257, 2049, 152, 2),
    (10_000, 10_000, 152, 2), (50_000, 3_000, 7, 3), (1 << 20, 1 << 20, 152, 2),
    (3_000, 1 << 20, 152, 2), (1 << 20, 100, 152, 2),
])
def test_plan_partitions_units(lib, n, m, sms, ctas):
    from paper_1402_4986_gb300 import plan_forward
    plan = plan_forward(n, m, 2.0, "f32c", sm_count=sms, ctas_per_sm=ctas)
    QT, TB = plan["queries_per_cta"], plan["records_per_tile"]
    assert plan["query_tiles"] == -(-m // QT)
    assert plan["data_tiles"] == -(-n // TB)
    assert plan["units"] == plan["query_tiles"] * plan["data_tiles"]
    assert 1 <= plan["grid"] <= min(plan["units"], sms * ctas)
    assert plan["partial_slots"] == plan["query_tiles"] + plan["grid"] - 1
    if plan["units"] <= 2_000_000:
        owner, slots = _cover(plan)
        # every unit has exactly one owner and owners are non-decreasing
        assert np.all(np.diff(owner) >= 0)
        # the slot of each (query tile, CTA) piece is unique and in range
        assert max(slots) < plan["partial_slots"]
        pieces = {(u // plan["data_tiles"], owner[u]) for u in range(plan["units"])}
        assert len(pieces) == len(slots)
        per_tile = {}
        for qt, g in pieces:
            per_tile.setdefault(qt, set()).add(g)
        assert max(len(v) for v in per_tile.values()) == plan["max_pieces_per_query_tile"]
        # balance: every CTA sweeps floor or ceil of units / grid
        counts = np.bincount(owner, minlength=plan["grid"])
        assert counts.max() - counts.min() <= 1


def test_plan_f64_form(lib):
    from paper_1402_4986_gb300 import plan_forward
    plan = plan_forward(1 << 20, 1 << 15, 2.0, "f64", sm_count=152, ctas_per_sm=4)
    assert plan["queries_per_cta"] == plan["threads_per_cta"] * plan["queries_per_thread"]
    assert plan["workspace_bytes"] >= plan["data_tiles"] * plan["records_per_tile"] * 24


def test_split_arithmetic_matches_paper_example(lib):
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_split_example.json")))
    assert (g["n"] + g["threads"] - 1) // g["threads"] == g["per_thread"]
    from paper_1402_4986_gb300 import plan_forward
    # The same ceiling split cuts the data into tiles: a tile as wide as the
    # paper's block gives the paper's count.
    plan = plan_forward(g["n"], 1, 2.0, "f32c", sm_count=1, ctas_per_sm=1)
    assert plan["data_tiles"] == -(-g["n"] // plan["records_per_tile"])
    assert plan["data_tiles"] * plan["records_per_tile"] >= g["n"] > \
        (plan["data_tiles"] - 1) * plan["records_per_tile"]


@pytest.mark.parametrize("bad", [dict(n=0), dict(m=-1), dict(p=0.0), dict(p=-2.0),
                                 dict(p=float("nan")), dict(p=float("inf")), dict(n=1 << 31)])
def test_plan_rejects_bad_arguments(lib, bad):
    from paper_1402_4986_gb300 import IDWError, plan_forward
    kw = dict(n=100, m=100, p=2.0)
    kw.update(bad)
    with pytest.raises(IDWError) as e:
        plan_forward(kw["n"], kw["m"], kw["p"])
    assert e.value.name == "IDW_ERR_INVALID_ARG"


def test_binding_rejects_host_tensors_for_device_entry():
    import torch
    import paper_1402_4986_gb300 as idw
    d = torch.zeros(4, 3)
    q = torch.zeros(2, 2)
    with pytest.raises(ValueError):
        idw.interpolate(d, q)
    with pytest.raises(ValueError):
        idw.interpolate(torch.zeros(4, 2), q)
    with pytest.raises(ValueError):
        idw.interpolate_local(d, q, 2.0, 0.1)
    with pytest.raises(ValueError):
        idw.interpolate_knn(d, q, 2.0, 4)
    with pytest.raises(ValueError):
        idw.LocalIndex(d, radius=0.1)
    with pytest.raises(ValueError):
        idw.LocalIndex(d, radius=0.1, k=4)
    with pytest.raises(ValueError):
        idw.interpolate_modified(d, q, 2.0, 0.1)
    with pytest.raises(ValueError):
        idw.local_backward(d, q, 2.0, 0.1, torch.ones(2))
    with pytest.raises(ValueError):
        idw.knn_backward(d, q, 2.0, 4, torch.ones(2))


# ------------------------------------------------- binding refusals (no GPU)
# The binding checks every caller-supplied buffer before it calls into the
# library, so a wrong size, dtype, device or layout raises ValueError instead
# of becoming an out-of-bounds device write or host read.

def _torch():
    return pytest.importorskip("torch")


def test_out_buffer_refusals():
    torch = _torch()
    import paper_1402_4986_gb300 as idw
    cpu = torch.device("cpu")
    ok = torch.empty(5)
    assert idw._check_buf(ok, 5, torch.float32, cpu, "out") is ok
    with pytest.raises(ValueError, match="hold 5 values"):
        idw._check_buf(torch.empty(4), 5, torch.float32, cpu, "out")        # too short
    with pytest.raises(ValueError, match="hold 5 values"):
        idw._check_buf(torch.empty(6), 5, torch.float32, cpu, "out")        # too long
    with pytest.raises(ValueError, match="float32"):
        idw._check_buf(torch.empty(5, dtype=torch.float64), 5, torch.float32, cpu, "out")
    with pytest.raises(ValueError, match="contiguous"):
        idw._check_buf(torch.empty(5, 2)[:, 0], 5, torch.float32, cpu, "out")
    with pytest.raises(ValueError, match="must be on cuda:0"):
        idw._check_buf(ok, 5, torch.float32, torch.device("cuda", 0), "out")  # wrong device
    with pytest.raises(ValueError, match="must be a tensor"):
        idw._check_buf([0.0] * 5, 5, torch.float32, cpu, "out")


def test_handle_device_refusal():
    torch = _torch()
    import paper_1402_4986_gb300 as idw

    class FakeHandle:
        device = 1
    h = FakeHandle()
    assert idw._handle_for(h, torch.device("cuda", 1)) is h
    with pytest.raises(ValueError, match="belongs to cuda:1"):
        idw._handle_for(h, torch.device("cuda", 0))
    with pytest.raises(ValueError, match="belongs to cuda:1"):
        idw._handle_for(h, torch.device("cpu"))


def test_upstream_gradient_refusals():
    torch = _torch()
    import paper_1402_4986_gb300 as idw
    cpu = torch.device("cpu")
    g = idw._grad_vec(torch.ones(3, 1, dtype=torch.float64), 3, cpu)
    assert g.dtype == torch.float32 and g.shape == (3,) and g.is_contiguous()
    with pytest.raises(ValueError, match="hold 3 values"):
        idw._grad_vec(torch.ones(2), 3, cpu)
    with pytest.raises(ValueError, match="tensor on cuda:0"):
        idw._grad_vec(torch.ones(3), 3, torch.device("cuda", 0))


def test_host_entry_point_shape_refusals():
    """interpolate_host reads n x 3 and m x 2 host values and writes m: a
    (n, 2) data array or a short out would be read or written out of bounds."""
    torch = _torch()
    import paper_1402_4986_gb300 as idw
    d = torch.zeros(8, 3)
    q = torch.zeros(5, 2)
    with pytest.raises(ValueError, match=r"data must be \(n, 3\)"):
        idw.interpolate_host(torch.zeros(8, 2), q)
    with pytest.raises(ValueError, match=r"queries must be \(m, 2\)"):
        idw.interpolate_host(d, torch.zeros(5, 3))
    with pytest.raises(ValueError, match="hold 5 values"):
        idw.interpolate_host(d, q, out=torch.empty(4))
    with pytest.raises(ValueError, match="float32"):
        idw.interpolate_host(d, q, out=torch.empty(5, dtype=torch.float64))
    with pytest.raises(ValueError, match="contiguous"):
        idw.interpolate_host(torch.zeros(3, 8).t(), q)
