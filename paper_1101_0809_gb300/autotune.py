"""Autotuner for the launch parameters of libpic: tile extents, particles per
thread block and sort interval.

Each candidate is timed on the caller's workload (device time per step, CUDA
events on the grid's stream, after warm-up) and the fastest is kept.  When the
sweep runs on a sample of the workload, the few fastest candidates can be timed
again on the whole of it (``refine``), and the fastest of those is kept.  Results
are cached per (workload key, device name) in a JSON file next to this module,
so that a later run of the same workload on the same kind of GPU skips the
sweep.
"""
import hashlib
import json
import os

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune_cache.json")


def workload_key(*parts):
    """Stable short hash of anything JSON-serialisable that defines the workload."""
    return hashlib.sha256(json.dumps(parts, sort_keys=True, default=str).encode()).hexdigest()[:16]


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(key, device, candidates, time_candidate, path=CACHE, refresh=False, refine=None, top=3):
    """Return (best, table, cached).

    ``candidates`` is a list of dicts of launch parameters; ``time_candidate(c)``
    builds the workload with them and returns milliseconds per step (or raises
    if the candidate is not valid for this workload, e.g. a tile too large for
    the smallest grid).  ``table`` lists (candidate, ms or None, reason).  With
    ``refine``, the ``top`` fastest candidates are timed again by ``refine(c)``
    and the fastest of those is the result; ``table`` then ends with those
    timings, marked "refined"."""
    db = _load(path)
    entry = f"{key}|{device}"
    if not refresh and entry in db:
        return db[entry]["best"], db[entry]["table"], True
    table = []
    for c in candidates:
        try:
            ms = float(time_candidate(c))
        except Exception as exc:          # an invalid candidate is skipped, with the reason
            table.append((c, None, str(exc)[:120]))
            continue
        table.append((c, ms, ""))
    valid = [t for t in table if t[1] is not None]
    if not valid:
        raise RuntimeError("no autotuning candidate ran: " + "; ".join(t[2] for t in table))
    best = min(valid, key=lambda t: t[1])[0]
    if refine is not None:
        final = []
        for c, _, _ in sorted(valid, key=lambda t: t[1])[:top]:
            try:
                ms = float(refine(c))
            except Exception as exc:
                table.append((c, None, "refined: " + str(exc)[:110]))
                continue
            table.append((c, ms, "refined"))
            final.append((c, ms))
        if final:
            best = min(final, key=lambda t: t[1])[0]
    db = _load(path)
    db[entry] = {"best": best, "table": table}
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1)
    os.replace(tmp, path)
    return best, table, False
