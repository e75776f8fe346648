// Full-plane spectrum path, float64 instantiation.
#include "gal_plane.cuh"
template struct gal::Plane<double>;
