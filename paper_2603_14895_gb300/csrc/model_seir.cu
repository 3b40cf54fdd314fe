// model_seir.cu -- row kernels of the SEIR model (one translation unit per model so that the
// template instantiations compile in parallel).
#include "rows.cuh"

namespace fsgp {
template int launch_rows<FSGP_SEIR>(const StepArgs &, const StepLaunch &, cudaStream_t);
template int occupancy_rows<FSGP_SEIR>(int, int, size_t, RowOccupancy *);
template int launch_split_rows<FSGP_SEIR>(const StepArgs &, int, int, int, int, cudaStream_t);
template int launch_persist<FSGP_SEIR>(const StepArgs &, const PersistArgs &, int, int, size_t, int, cudaStream_t, int *);
}  // namespace fsgp
