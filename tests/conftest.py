import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libvoge.so")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_terminal_summary(terminalreporter):
    """Lists that differ from the oracle's at allowed FP32/FP64 ties, per
    forward check, and each forward and gradient check's margins."""
    try:
        from parity import FWD_ERRS, GRAD_STATS, LIST_DIFFS
    except Exception:  # pragma: no cover
        return
    tr = terminalreporter
    if LIST_DIFFS:
        tr.section("index lists differing at allowed ties")
        for name, n_diff, total in LIST_DIFFS:
            tr.write_line(f"{n_diff:6d} of {total:8d}  {name}")
    if FWD_ERRS:
        tr.section("forward parity: worst |image - oracle| and |W - oracle| (bound 1e-4)")
        for name, ei, ew in FWD_ERRS:
            tr.write_line(f"{ei:9.2e} {ew:9.2e}  {name}")
    if GRAD_STATS:
        tr.section("gradient parity: relative norm error (bound 1e-3), worst per-element error / its bound")
        for name, key, rel, exc in GRAD_STATS:
            tr.write_line(f"{rel:9.2e} {exc:9.3f}  {key:10s} {name}")
