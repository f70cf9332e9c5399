"""Adaptive choice between the prior and Jacobi preconditioners (Sec. 3: the
better of the two can be picked for a given posterior at negligible cost by
comparing their performance every 100 Gibbs iterations).

A host-side policy, not arithmetic: it holds one library context per
preconditioner and decides which one serves each Gibbs step.  At every
`period`-th step it runs that step's draw with both and keeps the result of
the faster; the winner then serves the steps up to the next comparison.  The
draws themselves run in the library's kernels.
"""
from __future__ import annotations

import time
from typing import Callable, Dict, Optional

CHOICES = ("prior", "jacobi")


class AdaptivePreconditioner:
    """make_context(name) -> a library Context with that preconditioner;
    period: Gibbs steps between comparisons (the paper suggests 100);
    clock: a function returning seconds after the device has finished (the
    default synchronises CUDA around time.perf_counter)."""

    def __init__(self, make_context: Callable[[str], object], period: int = 100,
                 clock: Optional[Callable[[], float]] = None):
        if period < 1:
            raise ValueError("period must be at least 1")
        self.contexts: Dict[str, object] = {name: make_context(name) for name in CHOICES}
        self.period = int(period)
        self.current = "prior"
        self.history = []          # (step, {name: seconds}, chosen)
        self._clock = clock or _synced_clock

    def context(self) -> object:
        return self.contexts[self.current]

    def run(self, step: int, draw: Callable[[object], object]):
        """Runs draw(ctx) for Gibbs step `step` and returns its result.  On a
        comparison step both preconditioners draw (the same inputs, so either
        result is a valid draw) and the faster one's result is returned."""
        if step % self.period != 0:
            return draw(self.contexts[self.current])
        times, results = {}, {}
        for name in CHOICES:
            t0 = self._clock()
            results[name] = draw(self.contexts[name])
            times[name] = self._clock() - t0
        self.current = min(CHOICES, key=lambda n: times[n])
        self.history.append((step, times, self.current))
        return results[self.current]


def _synced_clock() -> float:
    import torch
    if torch.cuda.is_available():
        torch.cuda.synchronize()
    return time.perf_counter()
