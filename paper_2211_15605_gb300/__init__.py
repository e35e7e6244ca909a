"""GB300-native MP-PIC parcel-grid coupling step (Woo et al., arXiv 2211.15605, Sec. 2.1).

The compute path is the CUDA library ``libmppic`` (C ABI, declared in
``include/mppic.h``); :mod:`paper_2211_15605_gb300.mppic` is its thin Python
binding. Importing this package does not load the library; the first call into
the binding does, and raises if the library is missing.
"""
__all__ = ["mppic", "synth"]
