"""GB300-native multilevel fast multipole matvec for the boundary-integral block of
the coupled HDG-BI scattering solver (Zhao, Dong, Chen, Hu, Bagci; Sec. II.D-E).

Importing the package is cheap; the CUDA library is loaded on first use by
``paper_2210_04892_gb300.bi``.
"""
