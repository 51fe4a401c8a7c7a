// Band kernels instantiated for float (the two element types compile in parallel).
#define TPNS_BAND_PART 1
#include "kernels_band.cu"
