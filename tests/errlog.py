"""Achieved errors of the GPU parity tests, for the record: when the
environment variable CPH_ERROR_LOG names a file, every call appends one JSON
line {"case": ..., <metric>: <value>, ...} to it.  Nothing is written
otherwise; the tests' pass/fail bars do not depend on it."""
import json
import os


def record(case, **metrics):
    path = os.environ.get("CPH_ERROR_LOG")
    if not path:
        return
    line = {"case": case}
    line.update({k: (float(v) if hasattr(v, "__float__") else v) for k, v in metrics.items()})
    with open(path, "a") as f:
        f.write(json.dumps(line) + "\n")
