"""GB300-native dynamical perturbation theory (arXiv:2002.12872).

``paper_2002_12872_gb300.dpt`` binds the CUDA C-ABI library ``libdpt.so``;
``paper_2002_12872_gb300.inputs`` draws seeded synthetic problems.  Importing the
package itself loads nothing.
"""
