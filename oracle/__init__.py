"""CPU oracle for the pipe-flow time step (test infrastructure only)."""
