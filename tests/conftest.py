import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA device (parity tests of the CUDA path)")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle


def pytest_terminal_summary(terminalreporter):
    """Pixels compared with the oracle and, among them, pixels with a
    decision within single-precision reach of a threshold (each checked
    against the oracle's alternatives), per test."""
    tr = terminalreporter
    gb = sys.modules.get("test_gpu_backward")
    if gb is not None and getattr(gb, "GRAD_LOG", None):
        tr.write_sep("-", "gradient parity: entries within 1e-3 relative only through the floor")
        per = {}
        for case, name, n, floor_only in gb.GRAD_LOG:
            a = per.setdefault(name, [0, 0])
            a[0] += n
            a[1] += floor_only
        for name, (n, f) in per.items():
            tr.write_line(f"{name}: {f} of {n} entries ({f / max(n, 1):.2e})")
    gu = sys.modules.get("gpu_util")
    if gu is None or not getattr(gu, "FLAG_LOG", None):
        return
    per = {}
    for case, pix, flagged in gu.FLAG_LOG:
        a = per.setdefault(case, [0, 0, 0])
        a[0] += 1
        a[1] += pix
        a[2] += flagged
    tr.write_sep("-", "image parity: flagged pixels (checked against the oracle's alternatives)")
    tot = [0, 0]
    for case, (n, pix, flagged) in sorted(per.items()):
        tot[0] += pix
        tot[1] += flagged
        tr.write_line(f"{case}: {n} images, {pix} pixels, {flagged} flagged "
                      f"({flagged / max(pix, 1):.2e})")
    tr.write_line(f"total: {tot[0]} pixels, {tot[1]} flagged ({tot[1] / max(tot[0], 1):.2e})")
