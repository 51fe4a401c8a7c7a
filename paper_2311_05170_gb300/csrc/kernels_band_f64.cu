// Band kernels instantiated for double (the two element types compile in parallel).
#define TPNS_BAND_PART 2
#include "kernels_band.cu"
