"""Eq. 18 calibration constants, written by ``python -m oracle.calibrate --write``
(FP64 oracle on 1,000,000 core-shell primitives, seed 12345)."""
E_LN_GEM = -0.4889612576346142
E_COL = 0.008896804239666543
E_OPA = 0.1515067583205341
