"""GB300-native EBCC hot path: error-bounded two-layer (JPEG2000 + SPIHT)
compression of 2-D float32 fields, as CUDA kernels behind a C ABI
(include/ebcc.h).  The Python binding in `binding` only marshals arguments."""
