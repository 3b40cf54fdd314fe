// model_sisw.cu -- row kernels of SIS on weighted graphs (per-arc transmission draws;
// one translation unit per model so that the template instantiations compile in parallel).
#include "rows.cuh"

namespace fsgp {
template int launch_rows<kSisW>(const StepArgs &, const StepLaunch &, cudaStream_t);
template int occupancy_rows<kSisW>(int, int, size_t, RowOccupancy *);
template int launch_split_rows<kSisW>(const StepArgs &, int, int, int, int, cudaStream_t);
template int launch_persist<kSisW>(const StepArgs &, const PersistArgs &, int, int, size_t, int, cudaStream_t, int *);
}  // namespace fsgp
