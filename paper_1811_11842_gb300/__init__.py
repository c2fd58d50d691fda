"""GB300-native (sm_103a) solver for the per-time-step structured-grid linear
systems of the modified Cahn-Hilliard biofilm-flow model (McClanahan et al.,
§2-§4): the fourth-order phase-field system, the velocity-predictor systems
and the pressure Poisson system of the projection method.

Importing the package loads nothing; `binding` loads the CUDA library.
"""
