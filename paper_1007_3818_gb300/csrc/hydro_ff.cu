// hydro_ff.cu -- C-ABI entry points of the float-float mode (one translation
// unit per precision mode so the three instantiations compile in parallel).
#include "hydro_launch.cuh"

extern "C" int gamer_hydro_advance_ff(const float* in, float* out, float* face_flux,
                                      const double* dt, const double* dh, uint32_t* status,
                                      double* partials, int64_t N, const gh_params* p,
                                      void* stream) {
    return gamer::hydro_advance<GAMER_MODE_FF>(in, out, face_flux, dt, dh, status, partials, N, p,
                                          stream);
}

extern "C" int gamer_hydro_advance_level_ff(const float* level, float* out, float* face_flux,
                                            int32_t gx, int32_t gy, int32_t gz, int32_t bc,
                                            const double* dt, const double* dh,
                                            uint32_t* status, double* partials,
                                            const gh_params* p, void* stream) {
    return gamer::hydro_advance_level<GAMER_MODE_FF>(level, out, face_flux, gx, gy, gz, bc, dt, dh,
                                                status, partials, p, stream);
}

extern "C" int gamer_hydro_advance_level_window_ff(
    const float* window, float* out, float* face_flux, int32_t gx, int32_t gy, int32_t gz, int32_t bc,
    int32_t zb, int32_t zn, int32_t z0, int32_t nz, const double* dt, const double* dh,
    uint32_t* status, double* partials, const gh_params* p, void* stream) {
    return gamer::hydro_advance_level_window<GAMER_MODE_FF>(window, out, face_flux, gx, gy, gz, bc, zb, zn,
                                                  z0, nz, dt, dh, status, partials, p, stream);
}
