"""GB300 (sm_103a) greedy reduced-basis / column-pivoted QR library.

The compute path lives in the CUDA shared library built from ``csrc/``; the
Python side (``rb``) only marshals arguments through its C ABI.
"""
__version__ = "0.1.0"
