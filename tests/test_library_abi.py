"""The C-ABI library builds, loads and exports every symbol include/ddgs.h
declares (no GPU needed; no compute call is made)."""
import ctypes
import json
import os
import re

import pytest

from paper_2406_02518_gb300 import binding as B
from paper_2406_02518_gb300 import build as bld

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    bld.build()
    return B.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "ddgs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(ddgs_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_documented_entry_points():
    d = _declared()
    for n in ("ddgs_render", "ddgs_render_backward", "ddgs_workspace_create",
              "ddgs_workspace_destroy", "ddgs_debug_binning"):
        assert n in d


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(bld.LIB)
    for name in _declared():
        assert hasattr(raw, name), name
    assert sorted(B.EXPORTS) == _declared()


def test_parameter_count_matches_paper(lib):
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "parameter_count.json")))
    assert B.parameter_count(g["n_gaussians"], g["k"], g["L"]) == g["total_floats"]
    assert B.parameter_count(1, 8, 1) - B.parameter_count(0, 8, 1) == g["floats_per_gaussian"]
    assert B.parameter_count(0, 8, 1) == g["basis_floats"]
    assert B.parameter_count(-1, 8, 1) == -1


def test_status_strings(lib):
    lib.ddgs_status_string.restype = ctypes.c_char_p
    assert lib.ddgs_status_string(0) == b"ok"
    assert lib.ddgs_status_string(2) == b"pair capacity exceeded"


def test_null_arguments_are_rejected_without_a_gpu(lib):
    # argument validation happens on the host before any CUDA call
    assert lib.ddgs_render(None, None, None, None, None, None, None, None) == 1
    assert lib.ddgs_workspace_create(None) == 1
    assert lib.ddgs_l1_loss(None, None, 0, -1, 0, None, None, None) == 1


def test_binding_refuses_mis_shaped_tensors_before_any_call(lib):
    # the library takes raw pointers and sizes from the counts, so the binding
    # checks every tensor's shape and dtype on the host first
    import torch
    n = 5
    good = dict(means=torch.zeros(n, 3), log_scales=torch.zeros(n, 3), quats=torch.zeros(n, 4),
                opacity_logits=torch.zeros(n), feat_iso=torch.zeros(3, 8),
                feat_dir=torch.zeros(2, 8, dtype=torch.bfloat16), b_iso=torch.zeros(8),
                B_dir=torch.zeros(3, 8))
    B.Cloud(**good).validate()
    bad = [("means", torch.zeros(n, 2)), ("log_scales", torch.zeros(n, 3, dtype=torch.float64)),
           ("quats", torch.zeros(n, 3)), ("opacity_logits", torch.zeros(n, 1)),
           ("feat_iso", torch.zeros(3, 4)), ("feat_dir", torch.zeros(3, 8)),
           ("feat_dir", torch.zeros(2, 8, dtype=torch.float16)), ("b_iso", torch.zeros(1, 8)),
           ("B_dir", torch.zeros(4, 8)), ("B_dir", torch.zeros(3, 7))]
    for name, t in bad:
        with pytest.raises(ValueError, match=name):
            B.Cloud(**{**good, name: t}).validate()
    B.Views(torch.zeros(2, 3, 4), torch.zeros(2, 5), 8, 8).validate()
    with pytest.raises(ValueError, match="detector"):
        B.Views(torch.zeros(2, 3, 4), torch.zeros(1, 5), 8, 8).validate()
    with pytest.raises(ValueError, match="world_to_cam"):
        B.Views(torch.zeros(2, 12), torch.zeros(2, 5), 8, 8).validate()
    with pytest.raises(ValueError, match="target"):
        B.l1_loss(torch.zeros(2, 4, 4), torch.zeros(3, 4))


def test_batch_refuses_mis_shaped_requests(lib):
    import torch
    n = 4
    cloud = B.Cloud(torch.zeros(n, 3), torch.zeros(n, 3), torch.zeros(n, 4), torch.zeros(n),
                    torch.zeros(n, 8), torch.zeros(0, 8), torch.zeros(8), torch.zeros(3, 8))
    good = B.ViewGroup(torch.zeros(2, 3, 4), torch.zeros(2, 5), [(8, 8), (16, 4)])
    good.validate()
    with pytest.raises(ValueError, match="detector"):
        B.ViewGroup(torch.zeros(2, 3, 4), torch.zeros(3, 5), [(8, 8), (16, 4)]).validate()
    with pytest.raises(ValueError, match="clouds"):
        B.Batch([cloud, cloud], [good])
    bad_cloud = B.Cloud(torch.zeros(n, 3), torch.zeros(n, 3), torch.zeros(n, 4), torch.zeros(n + 1),
                        torch.zeros(n, 8), torch.zeros(0, 8), torch.zeros(8), torch.zeros(3, 8))
    with pytest.raises(ValueError, match="opacity_logits"):
        B.Batch([bad_cloud], [good])


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no CPU fallback: without the built library the binding raises
    monkeypatch.setattr(B, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        B.load(str(tmp_path / "libddgs.so"))
