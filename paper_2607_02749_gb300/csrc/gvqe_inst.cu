// gvqe_inst.cu -- explicit instantiation of the tile-pass kernels for one
// amplitude type and tile size, selected at compile time with
// -DGVQE_INST_T=<float|double> -DGVQE_INST_TB=<10..13>.  The build compiles
// this unit once per supported pair so the instantiations compile in parallel.
#include "gvqe_tile.cuh"

#if !defined(GVQE_INST_T) || !defined(GVQE_INST_TB)
#error "compile with -DGVQE_INST_T=float|double -DGVQE_INST_TB=10..13"
#endif

namespace gvqe {
template cudaError_t launch_tb<GVQE_INST_T, GVQE_INST_TB>(const PassArgs &, int, int, cudaStream_t);
}
