"""GB300-native SSW hot path: affine-gap Smith-Waterman-Gotoh alignment with
column maxima, secondary score, reversed-SW begin and banded CIGAR, as
hand-written CUDA for sm_103a behind a C ABI (``include/gsw.h``)."""
