"""GB300-native syndrome-based sum-product LDPC decoder with early termination.

The decoder itself is the CUDA library behind ``include/ldpc.h``; the Python
binding lives in ``paper_2507_03509_gb300.ldpc`` and loads it on import (it
raises if the library has not been built).  ``paper_2507_03509_gb300.gen``
holds the seeded synthetic inputs.
"""
