"""Geometries shared by the tests (tiny, both beams, odd and even sizes)."""
import numpy as np

from oracle import Geometry


def tiny_geometries():
    return [
        Geometry(beam=0, nx=8, ny=8, n_views=7, n_bins=11, angle_range=np.pi),
        Geometry(beam=0, nx=9, ny=7, n_views=12, n_bins=13, angle0=0.3, angle_range=2 * np.pi,
                 bin_pitch=0.8, det_offset=0.37),
        Geometry(beam=0, nx=16, ny=16, n_views=5, n_bins=23, angle0=0.1, angle_range=np.pi,
                 pixel=0.5, bin_pitch=0.45),
        Geometry(beam=1, nx=8, ny=8, n_views=9, n_bins=15, angle_range=2 * np.pi, bin_pitch=1.5,
                 src_to_center=20.0, src_to_det=30.0),
        Geometry(beam=1, nx=12, ny=10, n_views=10, n_bins=21, angle0=0.05, angle_range=2 * np.pi,
                 bin_pitch=1.2, det_offset=-0.4, src_to_center=11.0, src_to_det=19.0),
        Geometry(beam=1, nx=16, ny=16, n_views=6, n_bins=31, angle0=0.7, angle_range=2 * np.pi,
                 bin_pitch=1.0, src_to_center=14.0, src_to_det=21.0),
        # views at multiples of 45 degrees: driving-axis ties (|dir_x| = |dir_y| up to rounding)
        Geometry(beam=0, nx=8, ny=6, n_views=4, n_bins=13, angle_range=np.pi),
        Geometry(beam=1, nx=10, ny=10, n_views=8, n_bins=17, angle_range=2 * np.pi, bin_pitch=1.5,
                 src_to_center=25.0, src_to_det=37.5),
    ]
