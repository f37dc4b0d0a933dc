// step3d.cu -- placeholder until the 3D kernel lands.
#include "pf_internal.cuh"
namespace pf {
bool launch_step3d(int, int, int, int, int, cudaStream_t, const WorkItem*, int, const InstRec*, int) { return false; }
int occupancy_step3d(int, int, int, int) { return 0; }
}  // namespace pf
