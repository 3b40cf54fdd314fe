// model_ic.cu -- row kernels of the IC model (one translation unit per model so that the
// template instantiations compile in parallel).
#include "rows.cuh"

namespace fsgp {
template int launch_rows<FSGP_IC>(const StepArgs &, const StepLaunch &, cudaStream_t);
template int occupancy_rows<FSGP_IC>(int, int, size_t, RowOccupancy *);
template int launch_split_rows<FSGP_IC>(const StepArgs &, int, int, int, int, cudaStream_t);
template int launch_persist<FSGP_IC>(const StepArgs &, const PersistArgs &, int, int, size_t, int, cudaStream_t, int *);
}  // namespace fsgp
