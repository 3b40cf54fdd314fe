// model_sirw.cu -- row kernels of SIR on weighted graphs (per-arc transmission draws;
// one translation unit per model so that the template instantiations compile in parallel).
#include "rows.cuh"

namespace fsgp {
template int launch_rows<kSirW>(const StepArgs &, const StepLaunch &, cudaStream_t);
template int occupancy_rows<kSirW>(int, int, size_t, RowOccupancy *);
template int launch_split_rows<kSirW>(const StepArgs &, int, int, int, int, cudaStream_t);
template int launch_persist<kSirW>(const StepArgs &, const PersistArgs &, int, int, size_t, int, cudaStream_t, int *);
}  // namespace fsgp
