"""GB300-native DiaQ gate-apply path (arXiv 2405.01250).

The compute lives in the CUDA library libdiaq_gb300.so (include/diaq.h);
``paper_2405_01250_gb300.api`` is its thin PyTorch binding. Build the
library with ``paper_2405_01250_gb300.build.build()``.
"""
