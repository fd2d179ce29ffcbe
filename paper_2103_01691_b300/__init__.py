"""mu-mode integrator hot path on B300."""
