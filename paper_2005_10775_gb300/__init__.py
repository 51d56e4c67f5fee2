"""GB300-native nonlocal P1 stiffness assembly (D'Elia, Gunzburger, Vollmann).

Importing the package is cheap: the CUDA library is loaded on first use of
paper_2005_10775_gb300.nlfem.
"""
