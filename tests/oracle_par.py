"""Run the oracle on many tiles at once, on the host's cores.

The C oracle is single threaded and keeps no global state, and ctypes
releases the GIL while a foreign call runs, so independent oracle calls on
disjoint sets of requests run side by side in threads.  Each call still makes
its own pass over every object of the layer: this only spreads the requests,
it changes nothing the oracle computes.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np


def threads():
    return max(1, min(16, os.cpu_count() or 1))


def map_threads(fn, items, n_threads=None):
    """[fn(item) for item in items], evaluated in a thread pool."""
    with ThreadPoolExecutor(max_workers=n_threads or threads()) as ex:
        return list(ex.map(fn, items))


def render(render_fn, reqs, n_threads=None):
    """render_fn(reqs_chunk) -> (len(chunk), tile_bytes) uint8, evaluated on
    contiguous chunks of `reqs` in parallel and concatenated in order."""
    reqs = np.asarray(reqs)
    k = max(1, min(n_threads or threads(), len(reqs)))
    bounds = np.linspace(0, len(reqs), k + 1).astype(np.int64)
    chunks = [reqs[bounds[i]:bounds[i + 1]] for i in range(k) if bounds[i + 1] > bounds[i]]
    return np.concatenate(map_threads(render_fn, chunks, k))
