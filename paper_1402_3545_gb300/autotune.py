"""Autotuner cache: the Smooth tile variant chosen per level, kept in a JSON file keyed by GPU.

tune(op, prec) looks up (GPU name, grid shape, precision, whether lambda^2 varies) in the cache; on a
miss it runs the library's tpmg_autotune (which times every variant on the operator's own
workspace) and stores the result. The cache lives in $TPMG_TUNE_CACHE, else
~/.cache/tpmg/tuning.json. Only the schedule changes with the variant, never the per-cell
arithmetic.
"""
from __future__ import annotations

import json
import os

import torch

from . import tpmg


def cache_path() -> str:
    return os.environ.get("TPMG_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "tpmg", "tuning.json"))


def _load() -> dict:
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(d: dict) -> None:
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(d, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home directory only costs a re-tune next time


def key(operator: "tpmg.Operator", prec: int, lambda_varies: bool) -> str:
    gpu = torch.cuda.get_device_name(torch.cuda.current_device())
    return f"{gpu}|{operator.nx}x{operator.ny}x{operator.nz}|L{operator.L}|prec{prec}|var{int(lambda_varies)}"


def tune(operator: "tpmg.Operator", prec: int, lambda_varies: bool, reps: int = 5, force: bool = False) -> list[int]:
    """Variant per level (level 1 first), from the cache or measured now."""
    d = _load()
    k = key(operator, prec, lambda_varies)
    if not force and k in d and len(d[k]) == operator.L:
        choice = [int(x) for x in d[k]]
        for lvl, v in enumerate(choice, start=1):
            tpmg.set_variant(operator.op, prec, lvl, v)
        return choice
    choice = tpmg.autotune(operator.op, prec, operator.L, reps=reps)
    d[k] = choice
    _store(d)
    return choice
