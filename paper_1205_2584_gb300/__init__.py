"""GB300-native low-complexity damped Gauss-Newton (fLM) for dense CP.

The compute path lives in the C-ABI library built from ``csrc/`` and is
reached through ``paper_1205_2584_gb300.cpdgn`` (imported lazily so that
the input generator in ``synth`` can be used without a GPU).
"""
__all__ = ["synth", "cpdgn"]
