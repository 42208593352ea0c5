import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Right-hand-side parity figures of the run: plain relative L-infinity
    and the error relative to the term scale T, per comparison."""
    try:
        import parity
    except ImportError:
        return
    recs = parity.RECORDS
    if not recs:
        return
    tr = terminalreporter
    tr.section("right-hand-side parity (plain = |dR|/|R|, scaled = |dR|/max(|R|,T))")
    for r in recs:
        tr.write_line(f"{r['test']:<70s} {r['label']:<14s} N={r['N']:<2d} K={r['K']:<6d} "
                      f"plain={r['plain']:.2e} scaled={r['scaled']:.2e} T/|R|={r['T_over_R']:.3g}")
    worst = max(recs, key=lambda r: r["plain"])
    tr.write_line(f"worst plain {worst['plain']:.2e} ({worst['test']} {worst['label']}); "
                  f"worst scaled {max(r['scaled'] for r in recs):.2e}; "
                  f"{sum(r['plain'] > 1e-12 for r in recs)} of {len(recs)} above plain 1e-12")
    path = os.environ.get("PARITY_LOG")
    if path:
        with open(path, "w") as f:
            json.dump(recs, f, indent=1)
