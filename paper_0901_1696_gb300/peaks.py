"""GB300 unit counts used to state the FP64 roofline (the FP64 FMA pipe).

SM_COUNT and SM_MAX_MHZ are the part's (152 SMs on two dies, 2070 MHz
maximum SM clock).  FP64_FMA_PER_SM_CLK is the FP64 FMA issue rate per SM
per clock measured on GB300 with a DFMA throughput probe (1.196 TFLOP/s
at 2070 MHz, 95% of 2 FMA/clk/SM; profiles/fp_pipe_probe.md);
mma.sync f64 (DMMA) measured 1.049 TFLOP/s, below DFMA, so the FP64 pipe is
the roof.
"""
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
FP64_FMA_PER_SM_CLK = 2.0
# FP32 FMA issue rate per SM per clock (4 sub-partitions x 32 lanes); the
# same probe measured 74.46 TFLOP/s (118 FMA/clk/SM at 2070 MHz).
FP32_FMA_PER_SM_CLK = 128.0
