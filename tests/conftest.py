import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def write_report(name, text):
    """Report lines of the measurement tests go to the directory named by SFG_REPORT_DIR, if set."""
    d = os.environ.get("SFG_REPORT_DIR")
    if d and os.path.isdir(d):
        with open(os.path.join(d, name), "w") as fh:
            fh.write(text.rstrip("\n") + "\n")
