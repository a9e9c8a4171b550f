// Stand-ins for the forest storage functions the file parser (csrc/gf_io.cu) calls, so that the
// parser alone can be built with the host sanitizers and driven on CPU.  A file that passes every
// host check reaches gf_forest_alloc, which here reports GF_ENOMEM without touching a device.
#include "gf_internal.cuh"

#include <cstdarg>
#include <cstdio>
#include <string>

static thread_local std::string g_msg;

int gf_fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_msg = buf;
    return code;
}

int gf_cuda_fail(cudaError_t, const char *what) { return gf_fail(GF_ECUDA, "%s", what); }

extern "C" const char *gf_last_error(void) { return g_msg.c_str(); }

int gf_forest_alloc(gf_forest **out, const float *, int64_t, int32_t, int32_t, int32_t, bool, cudaStream_t) {
    *out = nullptr;
    return gf_fail(GF_ENOMEM, "stand-in: no device");
}

void gf_forest_destroy(gf_forest *) {}

int gf_forest_fill_structure(gf_forest *, const int32_t *, const float *, const int32_t *) { return GF_ENOMEM; }

int gf_forest_set_U(gf_forest *, const float *) { return GF_ENOMEM; }

extern "C" int gf_forest_add_screen(gf_forest *, int32_t, void *) { return GF_ENOMEM; }
