"""Seeded synthetic inputs (lung phantoms, blob and wave pairs) shared by the tests, the
smoke check and the benchmark.  Holds no registration arithmetic."""
from .generator import (FULL, SMALL, PhantomSpec, SplitMix64Stream, make_blob_pair,
                        make_lung_phantom, make_wave_pair, random_volume, true_field_mm)

__all__ = ["FULL", "SMALL", "PhantomSpec", "SplitMix64Stream", "make_blob_pair",
           "make_lung_phantom", "make_wave_pair", "random_volume", "true_field_mm"]
