"""GB300-native checkerboard-overrelaxation lattice gauge fixing (SU(2), SU(3)).

Import ``paper_1412_3655_gb300.culgt`` for the binding over the C-ABI library
``libculgt.so``; ``paper_1412_3655_gb300.synth`` generates seeded synthetic
gauge configurations. Importing the package itself loads nothing.
"""
