"""Regional (limited-area) domains used as test and benchmark inputs: a
projection name and the keyword arguments of ``Grid.regional`` /
``oracle.RegionalMesh`` (plane extents and projection parameters).  Plain
constants, no arithmetic of the method."""

# small domains of each projection (any nx, ny)
DOMAINS = {
    "rotated": ("rotated_lonlat", dict(xmin=-10.0, xmax=12.0, ymin=-8.0, ymax=9.0, south_pole=(10.0, -40.0))),
    "mercator": ("mercator", dict(xmin=-1.0e6, xmax=2.0e6, ymin=-5.0e5, ymax=3.0e6, lon0=20.0)),
    "lambert": ("lambert_conformal", dict(xmin=-1.0e6, xmax=1.0e6, ymin=-8.0e5, ymax=9.0e5, lat0=50.0, lon0=5.0)),
    "lambert_south": ("lambert_conformal",
                      dict(xmin=-1.2e6, xmax=9.0e5, ymin=-7.0e5, ymax=1.1e6, lat0=-35.0, lon0=140.0)),
    "polar": ("polar_stereographic", dict(xmin=-1.6e6, xmax=1.4e6, ymin=-1.5e6, ymax=1.5e6, lat0=90.0, lon0=-45.0)),
}

# a convection-permitting limited-area configuration: 1536 x 1440 points at
# 2.5 km on a Lambert conformal cone tangent at 46.5 N, 90 levels
LAM_NX, LAM_NY, LAM_NLEV = 1536, 1440, 90
LAM_DX = 2500.0
LAM = ("lambert_conformal",
       dict(xmin=-0.5 * (LAM_NX - 1) * LAM_DX, xmax=0.5 * (LAM_NX - 1) * LAM_DX,
            ymin=-0.5 * (LAM_NY - 1) * LAM_DX, ymax=0.5 * (LAM_NY - 1) * LAM_DX, lat0=46.5, lon0=2.0))
