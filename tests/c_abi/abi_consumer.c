/*
 * abi_consumer.c -- a plain C program using liblumipath through include/lumipath.h
 * alone (no Python), for the test suite.
 *
 *   abi_consumer check
 *       argument checks that need no GPU: every call returns a status, the
 *       message of the last failure is set, structure sizes agree with the header.
 *   abi_consumer render VIEWS.bin OUT.bin
 *       creates a 300 x 100 RGBA FP32 table (texel (i, j, c) =
 *       ((131 i + 71 j + 29 c) mod 1000) / 1000, exact in FP32), renders the
 *       lf_view structs of VIEWS.bin through lf_create_table / lf_render and
 *       writes the image ([P][4] float) and the indices ([P][10] int32) to OUT.bin.
 *
 * Exit status 0 on success; a failed check prints what failed and exits 1.
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "lumipath.h"

#define M_ORIGINS 300u
#define N_DIRECTIONS 100u

static int fails = 0;

static void expect(int ok, const char *what)
{
    if (!ok) {
        fprintf(stderr, "FAILED: %s (last error: %s)\n", what, lf_last_error());
        ++fails;
    }
}

static int check(void)
{
    expect(lf_version() != NULL && strlen(lf_version()) > 0, "lf_version");
    expect(lf_struct_size(0) == sizeof(lf_table_desc), "sizeof lf_table_desc");
    expect(lf_struct_size(1) == sizeof(lf_view), "sizeof lf_view");
    expect(lf_struct_size(2) == sizeof(lf_launch), "sizeof lf_launch");
    expect(lf_struct_size(3) == sizeof(lf_precompute_desc), "sizeof lf_precompute_desc");
    expect(lf_struct_size(4) == sizeof(lf_blob), "sizeof lf_blob");

    lf_table *t = (lf_table *)0x1;
    expect(lf_create_table(NULL, (const void *)0x1000, NULL, NULL, &t) == LF_ERR_INVALID_ARG, "NULL desc");
    expect(t == NULL, "output handle cleared on failure");
    expect(strlen(lf_last_error()) > 0, "error message set");

    lf_table_desc d;
    memset(&d, 0, sizeof d);
    d.radius = 1.0;
    d.n_origins = M_ORIGINS;
    d.n_directions = N_DIRECTIONS;
    d.channels = 2;
    d.dtype = LF_DTYPE_F32;
    expect(lf_create_table(&d, (const void *)0x1000, NULL, NULL, &t) == LF_ERR_INVALID_ARG, "channels = 2");
    d.channels = 4;
    d.radius = -1.0;
    expect(lf_create_table(&d, (const void *)0x1000, NULL, NULL, &t) == LF_ERR_INVALID_ARG, "radius < 0");
    d.radius = 1.0;
    d.dtype = LF_DTYPE_E4M3;
    expect(lf_create_table(&d, (const void *)0x1000, NULL, NULL, &t) == LF_ERR_INVALID_ARG, "E4M3 without scales");

    lf_view v;
    memset(&v, 0, sizeof v);
    expect(lf_render(NULL, &v, 1, (float *)0x1000, NULL, NULL) == LF_ERR_INVALID_ARG, "render without table");
    lf_destroy(NULL);

    const double c[3] = {0.0, 0.0, 0.0};
    float w[LF_POST_WEIGHTS];
    memset(w, 0, sizeof w);
    expect(lf_post_filter(1.0, c, 5, w, &v, 1, (const float *)0x1000, (float *)0x2000, NULL) == LF_ERR_INVALID_ARG,
           "post-filter channels = 5");
    if (fails == 0) printf("ok\n");
    return fails ? 1 : 0;
}

#define CUDA_OK(x)                                                                    \
    do {                                                                              \
        cudaError_t e_ = (x);                                                         \
        if (e_ != cudaSuccess) {                                                      \
            fprintf(stderr, "CUDA error %s at %s\n", cudaGetErrorString(e_), #x);    \
            return 1;                                                                 \
        }                                                                             \
    } while (0)

#define LF_OK_(x)                                                                     \
    do {                                                                              \
        lf_status s_ = (x);                                                           \
        if (s_ != LF_OK) {                                                            \
            fprintf(stderr, "lf error %d (%s) at %s\n", (int)s_, lf_last_error(), #x); \
            return 1;                                                                 \
        }                                                                             \
    } while (0)

static int render(const char *views_path, const char *out_path)
{
    FILE *f = fopen(views_path, "rb");
    if (!f) return 1;
    lf_view views[64];
    size_t nv = fread(views, sizeof(lf_view), 64, f);
    fclose(f);
    if (nv == 0) return 1;
    uint64_t P = 0;
    for (size_t k = 0; k < nv; ++k) {
        uint64_t end = views[k].out_offset + (uint64_t)views[k].width * views[k].height;
        if (end > P) P = end;
    }
    const size_t texels = (size_t)M_ORIGINS * N_DIRECTIONS * 4;
    float *host = (float *)malloc(texels * sizeof(float));
    for (uint32_t i = 0; i < M_ORIGINS; ++i)
        for (uint32_t j = 0; j < N_DIRECTIONS; ++j)
            for (uint32_t c = 0; c < 4; ++c)
                host[((size_t)i * N_DIRECTIONS + j) * 4 + c] = (float)((131u * i + 71u * j + 29u * c) % 1000u) / 1000.0f;
    float *table = NULL, *out = NULL;
    int32_t *idx = NULL;
    CUDA_OK(cudaMalloc((void **)&table, texels * sizeof(float)));
    CUDA_OK(cudaMemcpy(table, host, texels * sizeof(float), cudaMemcpyHostToDevice));
    CUDA_OK(cudaMalloc((void **)&out, P * 4 * sizeof(float)));
    CUDA_OK(cudaMalloc((void **)&idx, P * 10 * sizeof(int32_t)));

    lf_table_desc d;
    memset(&d, 0, sizeof d);
    d.radius = 1.0;
    d.n_origins = M_ORIGINS;
    d.n_directions = N_DIRECTIONS;
    d.channels = 4;
    d.dtype = LF_DTYPE_F32;
    lf_table *t = NULL;
    LF_OK_(lf_create_table(&d, table, NULL, NULL, &t));
    LF_OK_(lf_render(t, views, (uint32_t)nv, out, idx, NULL));
    LF_OK_(lf_sync_status(t, NULL));

    float *img = (float *)malloc(P * 4 * sizeof(float));
    int32_t *ix = (int32_t *)malloc(P * 10 * sizeof(int32_t));
    CUDA_OK(cudaMemcpy(img, out, P * 4 * sizeof(float), cudaMemcpyDeviceToHost));
    CUDA_OK(cudaMemcpy(ix, idx, P * 10 * sizeof(int32_t), cudaMemcpyDeviceToHost));
    lf_destroy(t);
    cudaFree(table);
    cudaFree(out);
    cudaFree(idx);
    f = fopen(out_path, "wb");
    if (!f) return 1;
    fwrite(img, sizeof(float), P * 4, f);
    fwrite(ix, sizeof(int32_t), P * 10, f);
    fclose(f);
    free(host);
    free(img);
    free(ix);
    printf("rendered %llu pixels\n", (unsigned long long)P);
    return 0;
}

int main(int argc, char **argv)
{
    if (argc >= 2 && strcmp(argv[1], "check") == 0) return check();
    if (argc >= 4 && strcmp(argv[1], "render") == 0) return render(argv[2], argv[3]);
    fprintf(stderr, "usage: abi_consumer check | render VIEWS.bin OUT.bin\n");
    return 2;
}
