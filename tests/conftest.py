import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


def pytest_terminal_summary(terminalreporter):
    """Worst element-wise ratio (error / tolerance) per compared quantity, when any ran."""
    try:
        import checks
    except ImportError:  # pragma: no cover
        return
    if checks.WORST:
        terminalreporter.write_line("element-wise parity, worst |error| / tolerance:")
        for k in sorted(checks.WORST):
            terminalreporter.write_line(f"  {k:32s} {checks.WORST[k]:.3g}")
