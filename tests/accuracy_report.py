"""Record of the achieved error of a GPU result against the FP64 oracle (or a closed
form), beside its gate.  Tests call ``record``; with the environment variable
MCRT_ACCURACY_OUT set to a file name, every record is appended to it as one JSON
line, so that a run of ``pytest -m gpu`` leaves the table of achieved errors.
"""
import json
import os


def record(config, quantity, value, gate, kind="max"):
    """config: workload name; quantity: what was measured; value: the measured error
    or fraction; gate: the bound the test asserts (None when only reported); kind:
    "max" when value must stay below gate, "min" when above."""
    path = os.environ.get("MCRT_ACCURACY_OUT")
    if not path:
        return
    with open(path, "a") as f:
        f.write(json.dumps({"config": config, "quantity": quantity, "value": float(value),
                            "gate": None if gate is None else float(gate), "kind": kind}) + "\n")


def integrated_error(gimgs, oimgs):
    """max over cameras and Stokes components of |sum X_gpu - sum X_oracle| / sum I_oracle."""
    return max(abs(g[e].sum() - o[e].sum()) / o[0].sum() for g, o in zip(gimgs, oimgs) for e in range(4))
