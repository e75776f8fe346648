// Full-plane spectrum path, float32 instantiation.
#include "gal_plane.cuh"
template struct gal::Plane<float>;
