// Volume kernel, launch shape of 128 threads per block, and the dispatch
// over the shapes (the kernel itself is in k_volume.cuh).
#include "k_volume.cuh"

SWE_VOLUME_SHAPE(128)

namespace swe {

void init_tables_volume() {
    volume_init_64();
    volume_init_128();
    volume_init_256();
}

void prepare_volume(swe_ctx* c) {
    volume_prepare_64(c->m.N);
    volume_prepare_128(c->m.N);
    volume_prepare_256(c->m.N);
}

bool volume_shape_valid(int N, int tpb) {
    if (tpb == 64) return volume_prepare_64(N);
    if (tpb == 128) return volume_prepare_128(N);
    if (tpb == 256) return volume_prepare_256(N);
    return false;
}

void launch_volume(swe_ctx* c, const double* W, double* R, cudaStream_t s, const int* stop) {
    if (c->p.volume == 1) {
        launch_volume_std(c, W, R, s, stop);
        return;
    }
    bool done = false;
    if (c->vol_tpb == 64) done = volume_launch_64(c, W, R, s, stop);
    else if (c->vol_tpb == 256) done = volume_launch_256(c, W, R, s, stop);
    if (!done) volume_launch_128(c, W, R, s, stop);
}

}  // namespace swe
