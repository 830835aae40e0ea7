"""Seeded synthetic workloads of the Fish School Behaviour step.

Input generators only: this module holds none of the method's arithmetic.
The initial fish state of every workload comes from the method's own
initialisation (Philox-keyed positions uniform over the pond, weight w0),
which the library and the oracle each implement; this module supplies the
sizes, seeds and step counts, and the ragged school sizes of the batched
ensemble (numpy's seeded generator, not the method's Philox).

The paper states neither the fish population nor the iteration count; the
sizes below are the ones the benchmark measures (C1..C5).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class SchoolWorkload:
    name: str
    n_fish: int
    seed: int
    steps: int
    school_id: int = 0


SMALL = SchoolWorkload("small N=10,000 T=100", 10_000, 0, 100)
RESIDENT = SchoolWorkload("resident N=2^20 T=1000", 1 << 20, 1, 1000)
STREAM = SchoolWorkload("stream N=2^28 T=100", 1 << 28, 2, 100)
# the stream school with the collective movements of fish-school search
# (collective_mode 1, volitive step 0.1)
COLLECTIVE = SchoolWorkload("collective N=2^28 T=100", 1 << 28, 2, 100)


@dataclass(frozen=True)
class BatchWorkload:
    name: str
    n_schools: int
    min_fish: int
    max_fish: int
    size_seed: int
    seed_base: int
    steps: int

    def sizes(self) -> np.ndarray:
        """School sizes, log-uniform in [min_fish, max_fish] (rounded)."""
        rng = np.random.default_rng(self.size_seed)
        u = rng.uniform(np.log(self.min_fish), np.log(self.max_fish), self.n_schools)
        return np.clip(np.rint(np.exp(u)), self.min_fish, self.max_fish).astype(np.uint64)

    def offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.sizes())]).astype(np.uint64)

    def seeds(self) -> np.ndarray:
        return (self.seed_base + np.arange(self.n_schools)).astype(np.uint64)


BATCH = BatchWorkload("batch 4096 schools N~logU[256,65536] T=500", 4096, 256, 65536,
                      size_seed=3, seed_base=1000, steps=500)

PRECISION = BatchWorkload("precision 64 schools x 2^24 T=1000", 64, 1 << 24, 1 << 24,
                          size_seed=0, seed_base=100, steps=1000)


def ragged_batch(n_schools: int, min_fish: int, max_fish: int, seed: int,
                 seed_base: int = 1000) -> BatchWorkload:
    """A smaller ragged ensemble of the same shape (tests)."""
    return BatchWorkload("ragged %d schools" % n_schools, n_schools, min_fish, max_fish,
                         size_seed=seed, seed_base=seed_base, steps=0)
