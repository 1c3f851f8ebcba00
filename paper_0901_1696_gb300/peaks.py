"""GB300 unit counts used to state the FP64 roofline (the FP64 FMA pipe).

SM_COUNT and SM_MAX_MHZ are the part's (152 SMs on two dies, 2070 MHz
maximum SM clock).  FP64_FMA_PER_SM_CLK is the FP64 FMA issue rate per SM
per clock measured on the GB300s with a DFMA throughput probe (see
profiles/fp64_peak_probe.md); mma.sync f64 (DMMA) was measured alongside.
"""
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
FP64_FMA_PER_SM_CLK = 2.0
