import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built extension")


# Parity results (whole-output relative L2 and the per-spectrum maximum of the
# same ratio) collected by the GPU tests; written as JSON lines to the path in
# PPF_PARITY_REPORT at the end of the session when that variable is set.
_PARITY = []


def record_parity(case: str, rel_l2: float, max_per_spectrum: float, tol: float) -> None:
    _PARITY.append({"case": case, "rel_l2": float(rel_l2), "max_per_spectrum": float(max_per_spectrum),
                    "tol": tol})


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("PPF_PARITY_REPORT")
    if path and _PARITY:
        import json
        with open(path, "w") as f:
            for r in _PARITY:
                f.write(json.dumps(r) + "\n")
