"""Persistent cache of batched-plan autotuning results (a JSON file).

fbf_plan_create autotunes by replaying every candidate schedule of the plan's
form on the given images and keeping the fastest.  For a batch seen before on
the same kind of GPU that choice is already known: the cache maps

    GPU name -> signature of the request -> {"schedule": name, "ms": ..., ...}

where the signature is a SHA-256 of the form, the border and, per image, its
shape, whether its rows meet TMA's 16-byte rules, and its filter parameters
(everything the candidate schedules and their speed depend on; not the
pointers or the pixel values).  A hit lets the plan capture the cached
schedule directly (fbf_plan_create_schedule, no replays); a miss autotunes and
records the choice.  Writes replace the file atomically (last writer wins).
The cache only ever changes which valid schedule runs, never the results.
"""
from __future__ import annotations

import hashlib
import json
import os
import tempfile

VERSION = 1

# filter parameters of an image spec that the signature covers, with defaults
_SPEC_KEYS = (("sigma_s", 3.0), ("W", 0), ("spatial", "gaussian"), ("range", "gaussian"), ("sigma_r", None),
              ("T", 255.0), ("eps", 1e-3), ("K_fixed", 0), ("levels", 0))


def signature(form: str, border: str, shapes, tma_ok, specs) -> str:
    """SHA-256 hex digest of a plan request: shapes are (H, W) per image,
    tma_ok whether its input rows meet TMA's 16-byte alignment rules."""
    imgs = []
    for (h, w), ok, sp in zip(shapes, tma_ok, specs):
        p = []
        for k, dflt in _SPEC_KEYS:
            v = sp.get(k, dflt)
            p.append(repr(float(v)) if isinstance(v, float) else v)
        imgs.append([int(h), int(w), bool(ok)] + p)
    blob = json.dumps({"v": VERSION, "form": form, "border": border, "images": imgs}, sort_keys=True,
                      separators=(",", ":"))
    return hashlib.sha256(blob.encode()).hexdigest()


def _load(path: str) -> dict:
    try:
        with open(path) as fh:
            d = json.load(fh)
        if isinstance(d, dict) and d.get("version") == VERSION and isinstance(d.get("entries"), dict):
            return d
    except (OSError, ValueError):
        pass
    return {"version": VERSION, "entries": {}}


def lookup(path: str, gpu: str, sig: str):
    """The cached entry (a dict with at least "schedule") or None."""
    e = _load(path)["entries"].get(gpu, {}).get(sig)
    return e if isinstance(e, dict) and isinstance(e.get("schedule"), str) else None


def record(path: str, gpu: str, sig: str, entry: dict) -> None:
    """Store `entry` under (gpu, sig), replacing the file atomically."""
    d = _load(path)
    d["entries"].setdefault(gpu, {})[sig] = entry
    folder = os.path.dirname(os.path.abspath(path))
    os.makedirs(folder, exist_ok=True)
    fd, tmp = tempfile.mkstemp(prefix=".fbf_tune_", dir=folder)
    try:
        with os.fdopen(fd, "w") as fh:
            json.dump(d, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        try:
            os.unlink(tmp)
        except OSError:
            pass
        raise
