/*
 * vt_oracle.h -- plain FP64 CPU Voronoi tessellator (test infrastructure only).
 *
 * Only tests, the smoke check and the benchmark's CPU-baseline leg may load
 * this library. The CUDA path neither includes this header nor links it.
 */
#ifndef VT_ORACLE_H
#define VT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    VTO_OK = 0,
    VTO_ERR_ARG = 1,        /* bad argument or a point outside [lo, hi) / not finite */
    VTO_ERR_DUPLICATE = 2,  /* two generators coincide: the cell is undefined */
    VTO_ERR_CAPACITY = 3    /* internal face / vertex capacity exceeded */
};

enum {
    VTO_MODE_SECURITY = 0,  /* kNN nearest first + security-radius stop + k doubling */
    VTO_MODE_BRUTE = 1      /* clip by every other generator, no stop test */
};

typedef struct vto_kdtree vto_kdtree;

/* Results for n_cells requested cells (in request order). All arrays are
 * owned by the result and released by vto_result_free. */
typedef struct {
    int64_t n_cells;
    int status;             /* first non-OK cell status, else VTO_OK */
    double* vol;            /* [n_cells] cell volume */
    double* cen;            /* [n_cells*3] centroid (global coordinates) */
    double* m2;             /* [n_cells] integral of |x - p_i|^2 over the cell */
    int64_t* nbr_off;       /* [n_cells+1] CSR offsets into nbr */
    int32_t* nbr;           /* neighbour generator indices, ascending per cell */
    int64_t n_nbr;
    int32_t* k_used;        /* [n_cells] k of the list that validated the cell */
    int32_t* n_clips;       /* [n_cells] bisectors that actually cut */
    int32_t* euler;         /* [n_cells] V - E + F of the final polyhedron */
    int32_t* nvert;         /* [n_cells] distinct vertices */
    int64_t* face_off;      /* [n_cells+1] CSR offsets into the face arrays */
    int32_t* face_tag;      /* generator index (>=0) or wall -1..-6 (x-,x+,y-,y+,z-,z+) */
    double* face_area;      /* face area */
    double* face_cen;       /* [F*3] face centroid (global) */
    double* face_plane;     /* [F*4] (n, b): n.(x - p_i) <= b */
    int32_t* face_size;     /* vertices per face */
    double* face_vtx;       /* [sum face_size * 3] CCW loops seen from outside (global); NULL unless geometry wanted */
    int64_t n_faces, n_face_vtx;
    int64_t* work_sign;     /* [n_cells] vertex-plane sign tests of the validating run */
    int64_t* work_newv;     /* [n_cells] vertices created by its cuts */
    int64_t* work_nbrs;     /* [n_cells] bisector planes it tested */
    int32_t* face_img;      /* image shift of each face's generator: (tx+2)*25 + (ty+2)*5 + (tz+2),
                               t in [-2, 2]^3; 62 (no shift) for every face of a non-periodic box */
    int periodic;           /* 1 for vto_tessellate_periodic */
} vto_result;

/* exact k nearest neighbours (self excluded) by (d2, index); missing slots get -1 / +inf */
int vto_knn(const float* pts, int64_t n, const int64_t* queries, int64_t nq, int k,
            int32_t* nbr, double* d2, int nthreads);

/* Voronoi cells of `cells` (all n when cells == NULL) inside the box [lo, hi).
 * order: optional permutation for VTO_MODE_BRUTE. */
int vto_tessellate(const float* pts, int64_t n, const float lo[3], const float hi[3],
                   int k0, int mode, const int64_t* order,
                   const int64_t* cells, int64_t n_cells, int want_geometry, int nthreads,
                   vto_result** result);

/* Periodic box [lo, hi) of periods L = hi - lo: every generator repeats at
 * p + t L. The cell of p_i starts as the cube [-L/2, L/2] around p_i; its
 * faces are tagged by generator (face_tag, p_i itself for the cube's faces)
 * and image shift (face_img); nbr lists the generator of every face, with
 * repeats when several images of one generator are faces. Requires
 * |L|^2 <= 4 min_a L_a^2 and n < 2^24 (else VTO_ERR_ARG). */
int vto_tessellate_periodic(const float* pts, int64_t n, const float lo[3], const float hi[3],
                            int k0, int mode, const int64_t* order,
                            const int64_t* cells, int64_t n_cells, int want_geometry, int nthreads,
                            vto_result** result);
/* exact k nearest images (own images excluded) by (d2, index, shift code) in
 * the periodic box; missing slots get -1 / -1 / +inf */
int vto_knn_periodic(const float* pts, int64_t n, const float lo[3], const float hi[3],
                     const int64_t* queries, int64_t nq, int k, int32_t* nbr, int32_t* img, double* d2,
                     int nthreads);
void vto_result_free(vto_result* r);

vto_kdtree* vto_kdtree_build(const float* pts, int64_t n);
void vto_kdtree_free(vto_kdtree* t);

#ifdef __cplusplus
}
#endif
#endif
