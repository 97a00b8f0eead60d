/*
 * orc_images.h -- TEST INFRASTRUCTURE ONLY (part of the FP64 reference).
 *
 * Table of image particles shared by the sphere and platelet references
 * (Section 2: periodic images added or removed as particles cross the
 * boundary, the alternative to the minimum image).  A particle in cell c of
 * an n-cell grid (0 <= c_a < n_a) has an image shifted by s_a L_a for every
 * combination of shifts s_a in {0} plus {+1 if c_a = 0} plus {-1 if c_a =
 * n_a - 1}, s != 0 -- the copies that lie within one cell of the box.  The
 * particle and its images are entries (id, s) of the grid padded by one cell
 * on every side (cells -1 .. n_a); entry (id, s) lies in padded cell
 * c + s n and stands for the point x_id + s L, formed when it is read.
 */
#ifndef ORC_IMAGES_H
#define ORC_IMAGES_H

#include <stdint.h>

typedef struct orc_imgtab {
    int dim;
    int64_t n[3];        /* cells per axis of the grid */
    double w[3];         /* cell widths */
    int64_t pn[3];       /* n + 2 per axis (1 for unused axes) */
    int64_t pcells;
    int64_t *cnt, *cap;  /* per padded cell: entries, room */
    int64_t **id;        /* per padded cell: particle ids */
    int8_t **sh;         /* per padded cell: 3 shifts per entry */
} orc_imgtab;

/* Entries of the N positions X (dim per particle) on the grid (n, w). */
void orc_imgtab_build(orc_imgtab *t, int dim, const int64_t n[3], const double w[3], const double *X, int64_t N);
/* Particle id moved from old to new: its entries follow. */
void orc_imgtab_move(orc_imgtab *t, int64_t id, const double *old, const double *new_);
/* Padded cell of position x's cell shifted by (dx, dy, dz) cells, dx..dz in
 * -1..1 (dz = 0 in 2D). */
int64_t orc_imgtab_near(const orc_imgtab *t, const double *x, int dx, int dy, int dz);
void orc_imgtab_free(orc_imgtab *t);
/* Mismatching padded cells between t and a rebuild from X (0: same). */
int64_t orc_imgtab_verify(orc_imgtab *t, const double *X, int64_t N);
/* Entries with a nonzero shift. */
int64_t orc_imgtab_images(const orc_imgtab *t);

#endif
